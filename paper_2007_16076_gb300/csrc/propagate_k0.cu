// Propagation kernels for the sum of grey levels (edge-cost kind 0), 4- and
// 8-connected.
#include "propagate.cuh"

namespace gapsp {

cudaError_t launch_k0(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st) {
    return conn == 8 ? launch_vpl<8, 0>(a, vpl, jobs, st) : launch_vpl<4, 0>(a, vpl, jobs, st);
}

}  // namespace gapsp
