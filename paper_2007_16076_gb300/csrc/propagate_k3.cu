// Propagation kernels for the sum over the channels of a multichannel image (edge-cost kind 3), 4- and
// 8-connected.
#include "propagate.cuh"

namespace gapsp {

cudaError_t launch_k3(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st) {
    return conn == 8 ? launch_vpl<8, 3>(a, vpl, jobs, st) : launch_vpl<4, 3>(a, vpl, jobs, st);
}

}  // namespace gapsp
