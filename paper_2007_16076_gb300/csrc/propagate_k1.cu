// Propagation kernels for the obstacle mask (edge-cost kind 1), 4- and
// 8-connected.
#include "propagate.cuh"

namespace gapsp {

cudaError_t launch_k1(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st) {
    return conn == 8 ? launch_vpl<8, 1>(a, vpl, jobs, st) : launch_vpl<4, 1>(a, vpl, jobs, st);
}

}  // namespace gapsp
