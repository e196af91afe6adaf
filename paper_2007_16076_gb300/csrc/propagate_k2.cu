// Propagation kernels for the L1 pseudo-metric (edge-cost kind 2), 4- and
// 8-connected.
#include "propagate.cuh"

namespace gapsp {

cudaError_t launch_k2(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st) {
    return conn == 8 ? launch_vpl<8, 2>(a, vpl, jobs, st) : launch_vpl<4, 2>(a, vpl, jobs, st);
}

}  // namespace gapsp
