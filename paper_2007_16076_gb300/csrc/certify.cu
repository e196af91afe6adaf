// Certificate of a result: every entry of every row checked against the
// equations that only the true distances satisfy.
//
// With positive integer edge weights, the geodesic distances from p are the
// unique solution of d(p,p) = 0 and, for r != p, d(p,r) = min over the
// neighbours q of r of d(p,q) + w(q,r) (Sec. 2, eqs. "temps" and
// "distance": a shortest path to r ends with an edge from a neighbour),
// the minimum over no reachable neighbour being "unreachable". Any other
// array breaks the equation somewhere: an entry too small has no neighbour
// to come from, an entry too large is beaten by one. So one pass that checks
// every entry against its neighbours in the same row proves the whole row
// exact, whatever computed it. Each thread checks one entry; the row's
// neighbouring entries are read through L1, the array once from DRAM.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gapsp {

namespace {

__device__ __forceinline__ int level(const CertifyArgs& a, int p) {
    return a.kind == 3 ? (int)__ldg(reinterpret_cast<const uint16_t*>(a.f) + p) : (int)__ldg(a.f + p);
}

__global__ void k_certify(CertifyArgs a) {
    const size_t n = (size_t)a.rows * a.N;
    unsigned long long bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / a.N), r = (int)(i - (size_t)k * a.N);
        const int p = a.src ? a.src[k] : k;
        const uint32_t* row = a.D + (size_t)k * a.N;
        const uint32_t v = __ldg(row + r);
        uint32_t want;
        if (r == p) {
            want = 0;
        } else if (a.kind == 1 && (!a.f[r] || !a.f[p])) {
            want = UNREACH;  // an obstacle joins nothing
        } else {
            const int rr = r / a.W, rc = r - rr * a.W;
            const int fr = a.kind == 1 ? 0 : level(a, r);
            uint64_t best = UNREACH;
            for (int dr = -1; dr <= 1; ++dr)
                for (int dc = -1; dc <= 1; ++dc) {
                    if (!dr && !dc) continue;
                    if (a.conn == 4 && dr && dc) continue;
                    const int qr = rr + dr, qc = rc + dc;
                    if (qr < 0 || qr >= a.H || qc < 0 || qc >= a.W) continue;
                    const int q = qr * a.W + qc;
                    if (a.kind == 1 && !a.f[q]) continue;
                    const uint32_t dq = __ldg(row + q);
                    if (dq == UNREACH) continue;
                    const int fq = a.kind == 1 ? 0 : level(a, q);
                    const uint32_t w = a.kind == 1 ? 2u : a.kind == 2 ? (uint32_t)(abs(fq - fr) + 1) : (uint32_t)(fq + fr + 1);
                    best = min(best, (uint64_t)dq + w);
                }
            want = (uint32_t)best;
        }
        bad += v != want;
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(FULL, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(a.bad, bad);
}

}  // namespace

cudaError_t launch_certify(const CertifyArgs& a, cudaStream_t st) {
    if (a.rows <= 0) return cudaSuccess;
    const size_t n = (size_t)a.rows * a.N;
    const size_t blocks = std::min<size_t>((n + 255) / 256, (size_t)152 * 16);
    k_certify<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gapsp
