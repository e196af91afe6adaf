// Kernels (a') and (b): the geodesic tree of each propagation and the fill of
// the distances array by Property 1 (Sec. 2).
//
// Tree. The paper leaves the choice of shortest-path tree open (Sec. 2,
// "geodesic tree"). Here every reached vertex b != s takes as parent its
// smallest-index neighbour q with d(s,q) + w(q,b) = d(s,b), read off the
// converged distances, so the tree does not depend on the relaxation order.
//
// Fill. For every reached b and every proper ancestor a of b,
// d(a,b) = d(s,b) - d(s,a) (Property 1). The pair is written into D (both
// triangles) the first time it is seen, and the fill counts cnt (Sec. 2, eq.
// "filling rate pt": tau(x) = (cnt(x) - 1)/(N - 1)) go up by one at both
// ends. "Distance operations" count every (ancestor, vertex) pair visited.
//
// To avoid visiting ancestors one by one, each tree path is cut into
// segments that stay inside one 8x8 pixel tile: for every vertex a,
// seg_mask(a) holds the bits of a and of its ancestors up to the first one
// outside a's tile, and seg_exit(a) is that first outside ancestor. The
// marks use the same tiling (one 64-bit word per row and tile), so one
// segment is tested against row b's marks with a single AND.
#include "common.cuh"
#include "internal.h"

namespace gapsp {

namespace {

__device__ __forceinline__ int edge_w(const TreeArgs& a, int p, int q) {
    return a.kind == 0 ? (int)a.f[p] + (int)a.f[q] + 1 : 2;
}

// parent[j][b] (-1 for the root and for unreached vertices).
__global__ void k_parents(TreeArgs a) {
    const int j = blockIdx.y;
    if (j >= *a.nsel) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.N) return;
    const int s = a.sel[j];
    const uint32_t* drow = a.D + (size_t)s * a.N;
    const uint32_t db = drow[b];
    int par = -1;
    if (b != s && db != UNREACH) {
        const int r = b / a.W, c = b - r * a.W;
        // neighbours in increasing linear index
        for (int dr = -1; dr <= 1 && par < 0; ++dr)
            for (int dc = -1; dc <= 1; ++dc) {
                if (!dr && !dc) continue;
                if (a.conn == 4 && dr && dc) continue;
                const int rr = r + dr, cc = c + dc;
                if (rr < 0 || rr >= a.H || cc < 0 || cc >= a.W) continue;
                const int q = rr * a.W + cc;
                if (a.kind == 1 && !a.f[q]) continue;
                const uint32_t dq = drow[q];
                if (dq != UNREACH && dq + (uint32_t)edge_w(a, q, b) == db) { par = q; break; }
            }
    }
    a.parent[(size_t)j * a.N + b] = par;
}

// seg_mask / seg_exit of every vertex of every selected tree.
__global__ void k_segments(TreeArgs a) {
    const int j = blockIdx.y;
    if (j >= *a.nsel) return;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.N) return;
    const TileGeom tg{a.W, a.tiles_w, a.words};
    const int32_t* par = a.parent + (size_t)j * a.N;
    const int t = tg.tile_of(v);
    unsigned long long m = 1ull << tg.bit_of(v);
    int x = par[v];
    for (int guard = 0; x >= 0 && guard < 64 && tg.tile_of(x) == t; ++guard) {
        m |= 1ull << tg.bit_of(x);
        x = par[x];
    }
    a.seg_mask[(size_t)j * a.N + v] = m;
    a.seg_exit[(size_t)j * a.N + v] = x;
}

// One block owns rows [b0, b0 + rows) of the marks, copied to shared memory,
// and walks, for each selected source, the tree path of each of its rows.
__global__ void k_fill(TreeArgs a) {
    extern __shared__ unsigned long long srow[];
    const int nsel = *a.nsel;
    if (nsel == 0) return;
    const int b0 = blockIdx.x * a.rows_per_block;
    const int nrows = min(a.rows_per_block, a.N - b0);
    const TileGeom tg{a.W, a.tiles_w, a.words};
    const unsigned long long* grow = a.marks + (size_t)b0 * a.words;
    for (int i = threadIdx.x; i < nrows * a.words; i += blockDim.x) srow[i] = ld_cg64(grow + i);
    __syncthreads();
    unsigned long long ops = 0, fresh = 0;
    const int items = nrows * nsel;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / nrows, bl = it - j * nrows, b = b0 + bl;
        const int s = a.sel[j];
        const uint32_t* drow = a.D + (size_t)s * a.N;
        const uint32_t db = drow[b];
        if (b == s || db == UNREACH) continue;
        const bool filled = *((volatile const uint32_t*)(a.cnt + b)) == (uint32_t)a.N;
        const int32_t* sexit = a.seg_exit + (size_t)j * a.N;
        const unsigned long long* smask = a.seg_mask + (size_t)j * a.N;
        unsigned long long* myrow = srow + (size_t)bl * a.words;
        int v = a.parent[(size_t)j * a.N + b];
        for (int guard = 0; v >= 0 && guard <= a.N; ++guard) {
            const unsigned long long m = smask[v];
            const int nx = sexit[v];
            ops += __popcll(m);
            if (!filled) {
                const int t = tg.tile_of(v);
                unsigned long long nb = m & ~myrow[t];
                while (nb) {
                    const int bit = __ffsll((long long)nb) - 1;
                    nb &= nb - 1;
                    const int ap = tg.pixel_of(t, bit);
                    // The pair {ap, b} is claimed on its canonical bit: row
                    // min(ap, b), column max(ap, b). The first claimant fills it.
                    const int lo = min(ap, b), hi = max(ap, b);
                    const unsigned long long cbit = 1ull << tg.bit_of(hi);
                    const unsigned long long old =
                        atomicOr(a.marks + (size_t)lo * a.words + tg.tile_of(hi), cbit);
                    if (!(old & cbit)) {
                        atomicOr(a.marks + (size_t)hi * a.words + tg.tile_of(lo), 1ull << tg.bit_of(lo));
                        atomicAdd(a.cnt + ap, 1u);
                        atomicAdd(a.cnt + b, 1u);
                        const uint32_t val = db - drow[ap];
                        a.Dw[(size_t)ap * a.N + b] = val;
                        a.Dw[(size_t)b * a.N + ap] = val;
                        ++fresh;
                    }
                    atomicOr(myrow + t, 1ull << bit);
                }
            }
            v = nx;
        }
    }
    // block totals
    for (int o = 16; o > 0; o >>= 1) {
        ops += __shfl_down_sync(FULL, ops, o);
        fresh += __shfl_down_sync(FULL, fresh, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ops) atomicAdd(a.stats + S_OPS, ops);
        if (fresh) atomicAdd(a.stats + S_NEW, fresh);
    }
}

}  // namespace

cudaError_t launch_parents(const TreeArgs& a, int B, cudaStream_t st) {
    dim3 grid((a.N + 255) / 256, B);
    k_parents<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_segments(const TreeArgs& a, int B, cudaStream_t st) {
    dim3 grid((a.N + 255) / 256, B);
    k_segments<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fill(const TreeArgs& a, int B, cudaStream_t st) {
    (void)B;
    const size_t smem = (size_t)a.rows_per_block * a.words * sizeof(unsigned long long);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int grid = (a.N + a.rows_per_block - 1) / a.rows_per_block;
    k_fill<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gapsp
