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
// ends (the counts are recomputed from the marks of the rows that changed).
// "Distance operations" count every (ancestor, vertex) pair visited.
//
// To avoid visiting ancestors one by one, each tree path is cut into
// segments that stay inside one 8x8 pixel tile: for every vertex a, the
// segment record holds the bits of a and of its ancestors up to the first
// one outside a's tile, and that first outside ancestor with its tile. The
// marks use the same tiling (one 64-bit word per row and tile), so one
// segment is tested against row b's marks with a single AND. The operation
// count (every ancestor pair, marked or not) comes from the tree depths
// instead, so rows already filled are not walked at all.
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace gapsp {

namespace {

// Row of pixel p without a division: exact for p < 2^16 and W <= 256.
__device__ __forceinline__ int row_of(const TreeArgs& a, int p) {
    return a.wdiv ? (int)__umulhi((unsigned)p, a.wdiv) : p;
}

// Tile << 8 | bit of pixel p (the layout of the marks).
__device__ __forceinline__ uint32_t tile_bit(const TreeArgs& a, int p) {
    const int r = row_of(a, p), c = p - r * a.W;
    return ((uint32_t)((r >> 3) * a.tiles_w + (c >> 3)) << 8) | (uint32_t)(((r & 7) << 3) | (c & 7));
}

// Canonical parent of b in the tree of s (-1 for the root and unreached):
// the first neighbour q in increasing index with d(s,q) + w(q,b) = d(s,b).
// fs: the grey levels (grey) or free flags (mask), in shared or global memory.
template <class Lv>
__device__ __forceinline__ int canonical_parent(const TreeArgs& a, const uint32_t* drow, const Lv* fs, int s,
                                                int b) {
    const uint32_t db = drow[b];
    if (b == s || db == UNREACH) return -1;
    const int W = a.W;
    const int r = row_of(a, b), c = b - r * W;
    const int f_b = fs[b];
    // w(q,b): f(q) + f(b) + 1 (sum, of grey levels or of channels), |f(q) - f(b)| + 1 (L1), 2 (mask)
    auto tight = [&](int q) {
        if (a.kind == 1 && !fs[q]) return false;
        const uint32_t dq = drow[q];
        const int fq = fs[q];
        const uint32_t w = (a.kind == 0 || a.kind == 3) ? (uint32_t)(fq + f_b + 1)
                           : a.kind == 2                 ? (uint32_t)(abs(fq - f_b) + 1)
                                                         : 2u;
        return dq != UNREACH && dq + w == db;
    };
    if (r > 0 && r + 1 < a.H && c > 0 && c + 1 < W) {
        // interior pixel: no bounds tests
        if (a.conn == 8) {
            const int off[8] = {-W - 1, -W, -W + 1, -1, 1, W - 1, W, W + 1};
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (tight(b + off[i])) return b + off[i];
        } else {
            const int off[4] = {-W, -1, 1, W};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (tight(b + off[i])) return b + off[i];
        }
        return -1;
    }
    for (int dr = -1; dr <= 1; ++dr)
        for (int dc = -1; dc <= 1; ++dc) {
            if (!dr && !dc) continue;
            if (a.conn == 4 && dr && dc) continue;
            const int rr = r + dr, cc = c + dc;
            if (rr < 0 || rr >= a.H || cc < 0 || cc >= W) continue;
            if (tight(rr * W + cc)) return rr * W + cc;
        }
    return -1;
}

// The tree of one selected source, one block per source:
//  1. the canonical parent of every vertex;
//  2. seg[j][v]: x = bits of v and of its ancestors up to the first one
//     outside v's 8x8 tile, the segment's exit; y = exit + 1 (bits 0-16, 0
//     past the root), the exit's tile (bits 17-26), and the same for the exit
//     of the exit's segment (bits 27-43 and 44-53), so that a walk can fetch
//     two segments at once;
//  3. the distance operations of the tree: the sum over reached b != s of
//     depth(b), the number of proper ancestors of b. With acc(v) = number of
//     vertices from v up to the root, depth(b) = acc(parent(b)); acc is
//     summed along the segment chain by pointer jumping. When N <= 16384
//     (SMALL) the parents and the jumping arrays are 16-bit shared arrays;
//     otherwise they live in global scratch.
// Canonical parent with the staged levels `sf` (8-bit, or 16-bit for the
// channel sum): sf points at pixel 0 of the staged range's coordinates.
__device__ __forceinline__ int parent_of(const TreeArgs& a, const uint32_t* drow, const void* sf, int s, int b) {
    return a.kind == 3 ? canonical_parent(a, drow, static_cast<const uint16_t*>(sf), s, b)
                       : canonical_parent(a, drow, static_cast<const uint8_t*>(sf), s, b);
}

// Stages levels [base, base + S) of the image into sf (same width).
__device__ __forceinline__ void stage_levels(const TreeArgs& a, void* sf, int base, int S) {
    if (a.kind == 3) {
        const uint16_t* f = reinterpret_cast<const uint16_t*>(a.f);
        for (int v = threadIdx.x; v < S; v += blockDim.x) static_cast<uint16_t*>(sf)[v] = f[base + v];
    } else {
        for (int v = threadIdx.x; v < S; v += blockDim.x) static_cast<uint8_t*>(sf)[v] = a.f[base + v];
    }
}

__host__ __device__ inline int level_bytes(int kind) { return kind == 3 ? 2 : 1; }

template <bool SMALL>
__global__ void __launch_bounds__(1024) k_tree(TreeArgs a) {
    extern __shared__ uint16_t sdep[];
    pdl_wait();
    pdl_trigger();
    __shared__ int s_any[2];
    const int j = blockIdx.x, B = gridDim.x;
    // the number of trees handed to k_depths (also when there are none)
    if (SMALL && a.dep_exit && j == 0 && threadIdx.x == 0) *a.dep_count = *a.nsel;
    if (j >= *a.nsel) return;
    const int N = a.N, s = a.sel[j];
    const uint32_t* drow = a.D + (size_t)s * N;
    int32_t* par = a.parent + (size_t)j * N;
    ulonglong2* seg = a.seg + (size_t)j * N;
    // SMALL: the distance row and the image are staged in shared memory (the
    // row shares the space of the jumping arrays, used only later); spar =
    // parent + 1, 0 for the root, 0xFFFF for unreached vertices
    uint16_t* spar = sdep + 4 * N;
    if (SMALL) {
        uint32_t* srow = reinterpret_cast<uint32_t*>(sdep);
        uint8_t* sf = reinterpret_cast<uint8_t*>(sdep + 5 * N);
        if ((N & 15) == 0 && a.kind != 3) {
            // 16-byte loads: the row starts at s * N * 4 bytes, the image at 0
            for (int v = 4 * threadIdx.x; v < N; v += 4 * blockDim.x)
                *reinterpret_cast<uint4*>(srow + v) = __ldcg(reinterpret_cast<const uint4*>(drow + v));
            for (int v = 16 * threadIdx.x; v < N; v += 16 * blockDim.x)
                *reinterpret_cast<uint4*>(sf + v) = __ldg(reinterpret_cast<const uint4*>(a.f + v));
        } else {
            for (int v = threadIdx.x; v < N; v += blockDim.x) srow[v] = __ldcg(drow + v);
            stage_levels(a, sf, 0, N);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < N; b += blockDim.x) {
            const int pb = parent_of(a, srow, sf, s, b);
            spar[b] = srow[b] == UNREACH ? (uint16_t)0xFFFF : (uint16_t)(pb + 1);
        }
    } else {
        for (int b = threadIdx.x; b < N; b += blockDim.x) par[b] = parent_of(a, drow, a.f, s, b);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const uint32_t gv = tile_bit(a, v);
        const uint32_t t = gv >> 8;
        unsigned long long m = 1ull << (gv & 63);
        const int sv = SMALL ? (int)spar[v] : 0;
        int x = SMALL ? (sv == 0xFFFF ? -1 : sv - 1) : __ldcg(par + v);
        uint32_t gx = x >= 0 ? tile_bit(a, x) : 0;
        for (int guard = 0; x >= 0 && guard < 64 && (gx >> 8) == t; ++guard) {
            m |= 1ull << (gx & 63);
            x = SMALL ? (int)spar[x] - 1 : __ldcg(par + x);
            gx = x >= 0 ? tile_bit(a, x) : 0;
        }
        const bool reached = SMALL ? sv != 0xFFFF : drow[v] != UNREACH;
        reinterpret_cast<unsigned long long*>(seg + v)[0] = m;
        if (SMALL) {
            sdep[v] = reached ? (uint16_t)__popcll(m) : 0;                 // acc, buffer 0
            sdep[2 * N + v] = reached ? (uint16_t)(x + 1) : 0;            // jmp + 1, buffer 0
        } else {
            a.acc[(size_t)j * N + v] = reached ? __popcll(m) : 0;
            a.jmp[(size_t)j * N + v] = reached ? x : -1;
        }
    }
    if (threadIdx.x == 0) { s_any[0] = 0; s_any[1] = 0; }
    __syncthreads();
    // the segment exits one and two steps ahead, with their tiles (before the
    // jumping passes overwrite the exit arrays)
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const int e1 = SMALL ? (int)sdep[2 * N + v] - 1 : __ldcg(a.jmp + (size_t)j * N + v);
        int e2 = -1;
        if (e1 >= 0) e2 = SMALL ? (int)sdep[2 * N + e1] - 1 : __ldcg(a.jmp + (size_t)j * N + e1);
        unsigned long long y = 0;
        if (e1 >= 0) y = (unsigned long long)(e1 + 1) | ((unsigned long long)(tile_bit(a, e1) >> 8) << 17);
        if (e2 >= 0) y |= ((unsigned long long)(e2 + 1) << 27) | ((unsigned long long)(tile_bit(a, e2) >> 8) << 44);
        reinterpret_cast<unsigned long long*>(seg + v)[1] = y;
    }
    if (SMALL && a.dep_exit) {
        // the depth sums run later, off the round's critical path
        uint16_t* ex = a.dep_exit + (size_t)j * N;
        uint16_t* sz = a.dep_size + (size_t)j * N;
        for (int v = threadIdx.x; v < N; v += blockDim.x) {
            ex[v] = sdep[2 * N + v];
            sz[v] = sdep[v];
        }
        return;
    }
    // pointer jumping: acc(v) += acc(jmp(v)); jmp(v) = jmp(jmp(v))
    int cur = 0;
    for (int pass = 0; pass < 32; ++pass) {
        const int nx = cur ^ 1;
        int any = 0;
        for (int v = threadIdx.x; v < N; v += blockDim.x) {
            int j1, c;
            if (SMALL) {
                j1 = (int)sdep[2 * N + cur * N + v] - 1;
                c = sdep[cur * N + v];
            } else {
                j1 = __ldcg(a.jmp + (size_t)(cur * B + j) * N + v);
                c = __ldcg(a.acc + (size_t)(cur * B + j) * N + v);
            }
            int j2 = -1;
            if (j1 >= 0) {
                if (SMALL) {
                    j2 = (int)sdep[2 * N + cur * N + j1] - 1;
                    c += sdep[cur * N + j1];
                } else {
                    j2 = __ldcg(a.jmp + (size_t)(cur * B + j) * N + j1);
                    c += __ldcg(a.acc + (size_t)(cur * B + j) * N + j1);
                }
            }
            any |= j2 >= 0;
            if (SMALL) {
                sdep[nx * N + v] = (uint16_t)c;
                sdep[2 * N + nx * N + v] = (uint16_t)(j2 + 1);
            } else {
                a.acc[(size_t)(nx * B + j) * N + v] = c;
                a.jmp[(size_t)(nx * B + j) * N + v] = j2;
            }
        }
        if (any) s_any[pass & 1] = 1;
        __syncthreads();
        const bool more = s_any[pass & 1] != 0;
        if (threadIdx.x == 0) s_any[(pass + 1) & 1] = 0;
        cur = nx;
        if (!more) break;
        __syncthreads();
    }
    unsigned long long ops = 0;
    for (int b = threadIdx.x; b < N; b += blockDim.x) {
        const int sb = SMALL ? (int)spar[b] : 0;
        const int pb = SMALL ? (sb == 0xFFFF ? -1 : sb - 1) : __ldcg(par + b);
        if (pb >= 0)
            ops += SMALL ? (unsigned long long)sdep[cur * N + pb]
                         : (unsigned long long)__ldcg(a.acc + (size_t)(cur * B + j) * N + pb);
    }
    for (int o = 16; o > 0; o >>= 1) ops += __shfl_down_sync(FULL, ops, o);
    if ((threadIdx.x & 31) == 0 && ops) atomicAdd(a.stats + S_OPS, ops);
}

// The tree of one selected source on a cluster of C blocks (N <= 16384,
// depth sums left to k_depths): each block owns a strip of rows, cut at a
// multiple of 8 so that no 8x8 tile is split, with the rows next to its strip
// staged for the parent tests. The second exit of a segment chain may lie in
// another strip; it is read from that block's shared memory. Same results
// as k_tree.
struct TreeCLayout {
    int hs, smax, pmax;  // rows per strip (the last may be shorter or empty); staged, owned pixels
    size_t o_par;        // byte offset of the parents (after the staged row and levels)
    __host__ __device__ TreeCLayout(int H, int W, int C, int lvb) {
        hs = (((H + C - 1) / C + 7) / 8) * 8;
        smax = (hs + 2) * W;
        pmax = hs * W;
        o_par = ((size_t)smax * (4 + lvb) + 15) & ~(size_t)15;
    }
    __host__ __device__ size_t bytes() const { return o_par + (size_t)pmax * 6 + 16; }
};

template <int C>
__global__ void __launch_bounds__(1024) k_treeC(TreeArgs a) {
    extern __shared__ __align__(16) unsigned char smc[];
    pdl_wait();
    pdl_trigger();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int j = blockIdx.x / C;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.dep_count = *a.nsel;
    if (j >= *a.nsel) return;  // all blocks of the cluster leave together
    const int N = a.N, W = a.W, H = a.H, s = a.sel[j];
    const TreeCLayout L(H, W, C, level_bytes(a.kind));
    const int r0 = min(rank * L.hs, H), r1 = min(r0 + L.hs, H);
    const int hr0 = r0 > 0 ? r0 - 1 : 0, hr1 = r1 < H ? r1 + 1 : H;
    const int base = hr0 * W, S = r1 > r0 ? (hr1 - hr0) * W : 0;  // staged pixels [base, base + S)
    const int p0 = r0 * W, P = (r1 - r0) * W;                     // owned pixels [p0, p0 + P)
    uint32_t* srow = reinterpret_cast<uint32_t*>(smc);
    uint8_t* sf = smc + (size_t)L.smax * 4;
    uint16_t* spar = reinterpret_cast<uint16_t*>(smc + L.o_par);
    uint16_t* acc = spar + L.pmax;
    uint16_t* jx = acc + L.pmax;
    const uint32_t* drow = a.D + (size_t)s * N;
    ulonglong2* seg = a.seg + (size_t)j * N;
    for (int v = threadIdx.x; v < S; v += blockDim.x) srow[v] = __ldcg(drow + base + v);
    stage_levels(a, sf, base, S);
    __syncthreads();
    // parents of the owned pixels (neighbours within the staged rows)
    const uint32_t* drow_l = srow - base;
    const void* sf_l = sf - (size_t)base * level_bytes(a.kind);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int b = p0 + i;
        const int pb = parent_of(a, drow_l, sf_l, s, b);
        spar[i] = drow_l[b] == UNREACH ? (uint16_t)0xFFFF : (uint16_t)(pb + 1);
    }
    __syncthreads();
    // segments: a tile's pixels and their in-tile ancestors are all owned
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int v = p0 + i;
        const uint32_t gv = tile_bit(a, v);
        const uint32_t t = gv >> 8;
        unsigned long long m = 1ull << (gv & 63);
        const int sv = spar[i];
        int x = sv == 0xFFFF ? -1 : sv - 1;
        uint32_t gx = x >= 0 ? tile_bit(a, x) : 0;
        for (int guard = 0; x >= 0 && guard < 64 && (gx >> 8) == t; ++guard) {
            m |= 1ull << (gx & 63);
            x = (int)spar[x - p0] - 1;
            gx = x >= 0 ? tile_bit(a, x) : 0;
        }
        const bool reached = sv != 0xFFFF;
        reinterpret_cast<unsigned long long*>(seg + v)[0] = m;
        acc[i] = reached ? (uint16_t)__popcll(m) : 0;
        jx[i] = reached ? (uint16_t)(x + 1) : 0;
    }
    cl.sync();  // every strip's exits are complete
    const uint16_t* jx_of[C];
#pragma unroll
    for (int r = 0; r < C; ++r) jx_of[r] = cl.map_shared_rank(jx, r);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int v = p0 + i;
        const int e1 = (int)jx[i] - 1;
        int e2 = -1;
        if (e1 >= 0) {
            const int re = min(row_of(a, e1) / L.hs, C - 1);
            e2 = (int)jx_of[re][e1 - re * L.hs * W] - 1;
        }
        unsigned long long y = 0;
        if (e1 >= 0) y = (unsigned long long)(e1 + 1) | ((unsigned long long)(tile_bit(a, e1) >> 8) << 17);
        if (e2 >= 0) y |= ((unsigned long long)(e2 + 1) << 27) | ((unsigned long long)(tile_bit(a, e2) >> 8) << 44);
        reinterpret_cast<unsigned long long*>(seg + v)[1] = y;
        a.dep_exit[(size_t)j * N + v] = jx[i];
        a.dep_size[(size_t)j * N + v] = acc[i];
    }
    cl.sync();  // no block leaves while another may read its exits
}

// The tree of one selected source on a cluster of C blocks for larger images
// (N > 16384, up to 65536): the same strips, parents and records as
// k_treeC, with 32-bit parents and exits, and the depth sums done in place:
// pointer jumping over the segment exits, each block owning its strip's
// entries and reading the others' through distributed shared memory, one
// cluster barrier per jump. Only the vertices that are some segment's exit
// (the entries of segments) take part in the jumps; every other vertex adds
// its exit's sum once at the end. An exit is kept as (owning block << 20 |
// index in its strip) + 1. Shared memory: the staged D rows (later the
// second exit buffer), the staged image, the parents (later the second
// count buffer), the first count and exit buffers, the entry flags.
struct TreeWLayout {
    int hs, smax, pmax;
    size_t o_par;  // byte offset of the parents
    __host__ __device__ TreeWLayout(int H, int W, int C, int lvb) {
        hs = (((H + C - 1) / C + 7) / 8) * 8;
        smax = (hs + 2) * W;
        pmax = hs * W;
        o_par = ((size_t)smax * (4 + lvb) + 15) & ~(size_t)15;
    }
    __host__ __device__ size_t bytes() const { return o_par + (size_t)pmax * 13 + 16; }
};

template <int C>
__global__ void __launch_bounds__(1024) k_treeW(TreeArgs a) {
    extern __shared__ __align__(16) unsigned char smw[];
    __shared__ int s_more[2];
    pdl_wait();
    pdl_trigger();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int j = blockIdx.x / C;
    if (j >= *a.nsel) return;  // all blocks of the cluster leave together
    const int N = a.N, W = a.W, H = a.H, s = a.sel[j];
    const TreeWLayout L(H, W, C, level_bytes(a.kind));
    const int r0 = min(rank * L.hs, H), r1 = min(r0 + L.hs, H);
    const int hr0 = r0 > 0 ? r0 - 1 : 0, hr1 = r1 < H ? r1 + 1 : H;
    const int base = hr0 * W, S = r1 > r0 ? (hr1 - hr0) * W : 0;  // staged pixels [base, base + S)
    const int p0 = r0 * W, P = (r1 - r0) * W;                     // owned pixels [p0, p0 + P)
    const int span = L.hs * W;                                    // pixels per strip
    uint32_t* srow = reinterpret_cast<uint32_t*>(smw);
    uint8_t* sf = smw + (size_t)L.smax * 4;
    uint32_t* spar = reinterpret_cast<uint32_t*>(smw + L.o_par);
    uint32_t* accA = spar + L.pmax;
    uint32_t* jxA = accA + L.pmax;
    uint8_t* entry = reinterpret_cast<uint8_t*>(jxA + L.pmax);  // is some segment's exit
    uint32_t* accB = spar;  // the parents are not needed once the segments are done
    uint32_t* jxB = srow;   // nor the staged rows once the parents are
    const uint32_t* drow = a.D + (size_t)s * N;
    ulonglong2* seg = a.seg + (size_t)j * N;
    if (threadIdx.x == 0) { s_more[0] = 0; s_more[1] = 0; }
    for (int v = threadIdx.x; v < S; v += blockDim.x) srow[v] = __ldcg(drow + base + v);
    stage_levels(a, sf, base, S);
    for (int i = threadIdx.x; i < P; i += blockDim.x) entry[i] = 0;
    cl.sync();  // every strip's flags are clear before any block marks them
    // parents of the owned pixels (neighbours within the staged rows); parent
    // + 1, 0 for the root, all ones for unreached pixels
    const uint32_t* drow_l = srow - base;
    const void* sf_l = sf - (size_t)base * level_bytes(a.kind);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int b = p0 + i;
        const int pb = parent_of(a, drow_l, sf_l, s, b);
        spar[i] = drow_l[b] == UNREACH ? 0xFFFFFFFFu : (uint32_t)(pb + 1);
    }
    __syncthreads();
    // segments: a tile's pixels and their in-tile ancestors are all owned
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int v = p0 + i;
        const uint32_t gv = tile_bit(a, v);
        const uint32_t t = gv >> 8;
        unsigned long long m = 1ull << (gv & 63);
        const uint32_t sv = spar[i];
        int x = sv == 0xFFFFFFFFu ? -1 : (int)sv - 1;
        uint32_t gx = x >= 0 ? tile_bit(a, x) : 0;
        for (int guard = 0; x >= 0 && guard < 64 && (gx >> 8) == t; ++guard) {
            m |= 1ull << (gx & 63);
            x = (int)spar[x - p0] - 1;
            gx = x >= 0 ? tile_bit(a, x) : 0;
        }
        const bool reached = sv != 0xFFFFFFFFu;
        reinterpret_cast<unsigned long long*>(seg + v)[0] = m;
        accA[i] = reached ? (uint32_t)__popcll(m) : 0u;
        uint32_t jx = 0;
        if (reached && x >= 0) {
            const int re = min(row_of(a, x) / L.hs, C - 1);
            const int li = x - re * span;
            jx = ((uint32_t)re << 20 | (uint32_t)li) + 1u;
            cl.map_shared_rank(entry, re)[li] = 1;
        }
        jxA[i] = jx;
    }
    cl.sync();  // every strip's exits and entry flags are complete (and its parents dead)
    // the exits one and two segments ahead
    auto pixel = [&](uint32_t jx) { return (int)((jx - 1) >> 20) * span + (int)((jx - 1) & 0xFFFFFu); };
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int v = p0 + i;
        const uint32_t j1 = jxA[i];
        const int e1 = j1 ? pixel(j1) : -1;
        int e2 = -1;
        if (j1) {
            const uint32_t j2 = cl.map_shared_rank(jxA, (int)((j1 - 1) >> 20))[(j1 - 1) & 0xFFFFFu];
            e2 = j2 ? pixel(j2) : -1;
        }
        unsigned long long y = 0;
        if (e1 >= 0) y = (unsigned long long)(e1 + 1) | ((unsigned long long)(tile_bit(a, e1) >> 8) << 17);
        if (e2 >= 0) y |= ((unsigned long long)(e2 + 1) << 27) | ((unsigned long long)(tile_bit(a, e2) >> 8) << 44);
        reinterpret_cast<unsigned long long*>(seg + v)[1] = y;
    }
    // depth sums: acc(v) = vertices from v up to the root, summed along the
    // chain of segment exits by pointer jumping (A -> B -> A ...) over the
    // entries (an entry's exit is an entry too); the A buffers of the other
    // vertices keep their segment's count and exit for the last step
    int cur = 0;
    for (int pass = 0; pass < 32; ++pass) {
        uint32_t* ac = cur ? accB : accA;
        uint32_t* jc = cur ? jxB : jxA;
        uint32_t* an = cur ? accA : accB;
        uint32_t* jn = cur ? jxA : jxB;
        int any = 0;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            if (!entry[i]) continue;
            const uint32_t j1 = jc[i];
            uint32_t c = ac[i], j2 = 0;
            if (j1) {
                const int re = (int)((j1 - 1) >> 20), li = (int)((j1 - 1) & 0xFFFFFu);
                c += cl.map_shared_rank(ac, re)[li];
                j2 = cl.map_shared_rank(jc, re)[li];
            }
            any |= j2 != 0;
            an[i] = c;
            jn[i] = j2;
        }
        if (any) s_more[pass & 1] = 1;
        cl.sync();  // every strip has jumped once; no one reads the old buffers any more
        int more = 0;
#pragma unroll
        for (int r = 0; r < C; ++r) more |= *((volatile int*)cl.map_shared_rank(s_more + (pass & 1), r));
        if (threadIdx.x == 0) s_more[(pass + 1) & 1] = 0;
        cur ^= 1;
        __syncthreads();  // the flag of the next pass is clear before anyone sets it
        if (!more) break;
    }
    const uint32_t* af = cur ? accB : accA;
    unsigned long long ops = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        uint32_t c;
        if (entry[i]) {
            c = af[i];
        } else {
            // a segment's count plus its exit's sum (A still holds both)
            const uint32_t j1 = jxA[i];
            c = accA[i];
            if (j1) c += cl.map_shared_rank(af, (int)((j1 - 1) >> 20))[(j1 - 1) & 0xFFFFFu];
        }
        if (c > 1) ops += (unsigned long long)(c - 1);  // unreached vertices hold 0, the root 1
    }
    for (int o = 16; o > 0; o >>= 1) ops += __shfl_down_sync(FULL, ops, o);
    if ((threadIdx.x & 31) == 0 && ops) atomicAdd(a.stats + S_OPS, ops);
    cl.sync();  // no block leaves while another may read its shared memory
}

// Distance operations of one tree from its segment exits and sizes (N <=
// 16384): acc(v) = number of vertices from v up to the root, summed along
// the chain of segment exits by pointer jumping; depth(b) = acc(b) - 1.
__global__ void __launch_bounds__(1024) k_depths(TreeArgs a) {
    extern __shared__ uint16_t sd[];  // acc [2][N], exit + 1 [2][N]
    __shared__ int s_any[2];
    const int j = blockIdx.x;
    if (j >= *a.dep_count) return;
    const int N = a.N;
    const uint16_t* ex = a.dep_exit + (size_t)j * N;
    const uint16_t* sz = a.dep_size + (size_t)j * N;
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        sd[v] = sz[v];
        sd[2 * N + v] = ex[v];
    }
    if (threadIdx.x == 0) { s_any[0] = 0; s_any[1] = 0; }
    __syncthreads();
    int cur = 0;
    for (int pass = 0; pass < 32; ++pass) {
        const int nx = cur ^ 1;
        int any = 0;
        for (int v = threadIdx.x; v < N; v += blockDim.x) {
            const int j1 = (int)sd[2 * N + cur * N + v] - 1;
            int c = sd[cur * N + v], j2 = -1;
            if (j1 >= 0) {
                j2 = (int)sd[2 * N + cur * N + j1] - 1;
                c += sd[cur * N + j1];
            }
            any |= j2 >= 0;
            sd[nx * N + v] = (uint16_t)c;
            sd[2 * N + nx * N + v] = (uint16_t)(j2 + 1);
        }
        if (any) s_any[pass & 1] = 1;
        __syncthreads();
        const bool more = s_any[pass & 1] != 0;
        if (threadIdx.x == 0) s_any[(pass + 1) & 1] = 0;
        cur = nx;
        if (!more) break;
        __syncthreads();
    }
    unsigned long long ops = 0;
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const int c = sd[cur * N + v];
        if (c > 1) ops += (unsigned long long)(c - 1);  // unreached vertices hold 0, the root 1
    }
    for (int o = 16; o > 0; o >>= 1) ops += __shfl_down_sync(FULL, ops, o);
    if ((threadIdx.x & 31) == 0 && ops) atomicAdd(a.stats + S_OPS, ops);
}

// One block owns up to 32 consecutive rows of the marks. Rows already
// filled (cnt = N) hold every pair and are skipped; the others are copied
// to shared memory. For each selected source the block walks the tree path
// of each of its rows b, one tile segment at a time, from b's own segment
// record: ORing a segment into the shared copy of row b returns the bits it
// already had, and the others are new pairs {a, b}, so a pair that several
// trees of the round share is taken once per row. For every new pair,
// D[a][b] = D[b][a] = d(s,b) - d(s,a) (Property 1) and the mirror bit (row
// a, column b) is ORed into the global marks without waiting for the old
// value; the shared rows are ORed back at the end. A pair found from both of
// its rows in the same round is written twice with the same value; the
// counts come from the marks (k_recount), which hold each pair once per row.
__global__ void __launch_bounds__(256, 4) k_fill(TreeArgs a) {
    extern __shared__ unsigned long long srow[];
    pdl_wait();
    pdl_trigger();
    __shared__ int s_rows[32], s_tile[32], s_bit[32];
    __shared__ int s_nu;
    const int nsel = *a.nsel;
    if (nsel == 0) return;
    const int b0 = blockIdx.x * a.rows_per_block;
    const int nrows = min(a.rows_per_block, a.N - b0);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const bool open = lane < nrows && __ldcg(a.cnt + b0 + lane) < (uint32_t)a.N;
        const unsigned m = __ballot_sync(FULL, open);
        if (open) {
            const int i = __popc(m & ((1u << lane) - 1u));
            const uint32_t g = __ldg(a.pgeo + b0 + lane);
            s_rows[i] = b0 + lane;
            s_tile[i] = (int)(g >> 8);
            s_bit[i] = (int)(g & 63);
        }
        if (lane == 0) {
            s_nu = __popc(m);
        }
    }
    __syncthreads();
    const int nu = s_nu;
    if (nu == 0) return;
    const int words = a.words;
    // the shared rows are padded by one word (and their "changed" bytes by
    // four) so that the same tile of different rows falls in different banks
    const int rs = fill_row_stride(words), cs = fill_chg_stride(words);
    uint8_t* chg = reinterpret_cast<uint8_t*>(srow + (size_t)a.rows_per_block * rs);
    for (int i = threadIdx.x; i < nu * words; i += blockDim.x) {
        const int w = i / nu, r = i - w * nu;  // neighbouring threads: neighbouring rows, one tile
        srow[r * rs + w] = ld_cg64(a.marks + (size_t)w * a.N + s_rows[r]);
        chg[r * cs + w] = 0;
    }
    __syncthreads();
    const int items = nu * nsel;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / nu, bl = it - j * nu, b = s_rows[bl];
        const int s = a.sel[j];
        const uint32_t* drow = a.D + (size_t)s * a.N;
        const uint32_t db = __ldg(drow + b);
        if (b == s || db == UNREACH) continue;
        const ulonglong2* seg = a.seg + (size_t)j * a.N;
        unsigned long long* myrow = srow + (size_t)bl * rs;
        uint8_t* mychg = chg + (size_t)bl * cs;
        const int tb = s_tile[bl];
        const unsigned long long bbit = 1ull << s_bit[bl];
        // one tile segment: the bits of m not yet in row b are new pairs
        auto take = [&](int t, unsigned long long m) {
            // a plain read first: most segments bring nothing new, and the
            // shared-memory atomics are the scarce resource here
            unsigned* w32 = reinterpret_cast<unsigned*>(myrow + t);
            const unsigned lo = (unsigned)m & ~((volatile unsigned*)w32)[0];
            const unsigned hi = (unsigned)(m >> 32) & ~((volatile unsigned*)w32)[1];
            if (!(lo | hi)) return;
            // claim the bits that look new: two 32-bit ORs (a 64-bit OR on
            // shared memory is much slower); another tree of the round may
            // have set some of them meanwhile
            const unsigned olo = lo ? atomicOr(w32, lo) : 0xFFFFFFFFu;
            const unsigned ohi = hi ? atomicOr(w32 + 1, hi) : 0xFFFFFFFFu;
            unsigned long long nb = (((unsigned long long)hi << 32) | lo) & ~(((unsigned long long)ohi << 32) | olo);
            if (!nb) return;
            mychg[t] = 1;
            const int base = __ldg(a.tbase + t);
            // up to 8 new pairs at a time: the distance loads first, so that
            // they are in flight together, then the stores. The rows d(s, .)
            // read here only ever receive the same exact values again, so
            // read-only loads are safe.
            while (nb) {
                int ap[8];
                uint32_t dv[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    ap[k] = -1;
                    if (nb) {
                        const int bit = __ffsll((long long)nb) - 1;
                        nb &= nb - 1;
                        ap[k] = base + (bit >> 3) * a.W + (bit & 7);
                        dv[k] = __ldg(drow + ap[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (ap[k] < 0) continue;
                    const uint32_t val = db - dv[k];
                    atomicOr(a.marks + (size_t)tb * a.N + ap[k], bbit);
                    // streaming stores: D is far larger than L2, keep the
                    // trees and marks resident instead
                    __stcs(a.Dw + (size_t)ap[k] * a.N + b, val);
                    __stcs(a.Dw + (size_t)b * a.N + ap[k], val);
                }
            }
        };
        ulonglong2 g = __ldg(seg + b);
        unsigned long long m = g.x & ~bbit;  // b's ancestors inside b's tile
        int t = tb;
        for (int guard = 0; guard <= a.N; ++guard) {
            // the next two segments are fetched together, before this one is
            // worked on
            const unsigned long long y = g.y;
            const int e1 = (int)(y & 0x1FFFFu) - 1, t1 = (int)((y >> 17) & 0x3FFu);
            const int e2 = (int)((y >> 27) & 0x1FFFFu) - 1, t2 = (int)((y >> 44) & 0x3FFu);
            unsigned long long m1 = 0;
            ulonglong2 g2 = make_ulonglong2(0ull, 0ull);
            if (e1 >= 0) m1 = __ldg(reinterpret_cast<const unsigned long long*>(seg + e1));
            if (e2 >= 0) g2 = __ldg(seg + e2);
            take(t, m);
            if (e1 < 0) break;
            take(t1, m1);
            if (e2 < 0) break;
            g = g2;
            t = t2;
            m = g.x;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nu * words; i += blockDim.x) {
        const int w = i / nu, r = i - w * nu;
        if (chg[r * cs + w]) atomicOr(a.marks + (size_t)w * a.N + s_rows[r], srow[r * rs + w]);
    }
}

#ifndef FILL_G_MINB
#define FILL_G_MINB 8
#endif

// The same fill with the marks claimed in global memory, through L2: no
// staging, so a block needs no shared memory and no barrier, and every warp
// leaves as soon as its own walks end. A warp owns 8 consecutive rows
// (lanes 0-7, 8-15, ...: the same rows) for 4 trees, so the 8 walks of one
// tree, whose paths soon merge, fetch mostly the same records. Each step of
// a walk fetches together the next two segment masks, the record two
// segments ahead and row b's mark words for the two tiles of those
// segments; a segment's bits not yet in the word are claimed with one 64-bit
// atomic OR (the word read ahead may be stale, the OR's old value decides).
// A claimed bit is a new pair {a, b}: D[a][b] = D[b][a] = d(s,b) - d(s,a)
// (Property 1) and the mirror bit (row a, column b) as in k_fill.
__global__ void __launch_bounds__(128, FILL_G_MINB) k_fill_g(TreeArgs a, int quads) {
    pdl_wait();
    pdl_trigger();
    const int nsel = *a.nsel;
    if (nsel == 0) return;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int grp = warp / quads, quad = warp - grp * quads;
    const int b = grp * 8 + (lane & 7), j = quad * 4 + (lane >> 3);
    if (b >= a.N || j >= nsel) return;
    if (__ldcg(a.cnt + b) >= (uint32_t)a.N) return;  // row b holds every pair already
    const int s = a.sel[j];
    // 32-bit offsets (N^2 < 2^32): fewer registers, more warps in flight
    const uint32_t srow = (uint32_t)s * (uint32_t)a.N, brow = (uint32_t)b * (uint32_t)a.N;
    const uint32_t db = __ldg(a.D + srow + b);
    if (b == s || db == UNREACH) return;
    const ulonglong2* seg = a.seg + (size_t)j * a.N;
    unsigned long long* const mrow = a.marks + b;  // row b's word of tile t at mrow[t * N]
    const uint32_t gb = __ldg(a.pgeo + b);
    const int tb = (int)(gb >> 8);
    const unsigned long long bbit = 1ull << (gb & 63);
    auto take = [&](int t, unsigned long long m, unsigned long long w) {
        unsigned long long nb = m & ~w;
        if (!nb) return;
        nb &= ~atomicOr(mrow + (uint32_t)t * (uint32_t)a.N, nb);
        if (!nb) return;
        const int base = __ldg(a.tbase + t);
        while (nb) {
            int ap[4];
            uint32_t dv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ap[k] = -1;
                if (nb) {
                    const int bit = __ffsll((long long)nb) - 1;
                    nb &= nb - 1;
                    ap[k] = base + (bit >> 3) * a.W + (bit & 7);
                    dv[k] = __ldg(a.D + srow + ap[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (ap[k] < 0) continue;
                const uint32_t val = db - dv[k];
                atomicOr(a.marks + (uint32_t)tb * (uint32_t)a.N + ap[k], bbit);
                __stcs(a.Dw + (uint32_t)ap[k] * (uint32_t)a.N + b, val);
                __stcs(a.Dw + brow + ap[k], val);
            }
        }
    };
    ulonglong2 g = __ldg(seg + b);
    unsigned long long m = g.x & ~bbit;  // b's ancestors inside b's tile
    int t = tb;
    unsigned long long w = ld_cg64(mrow + (uint32_t)t * (uint32_t)a.N);
    for (int guard = 0; guard <= a.N; ++guard) {
        const unsigned long long y = g.y;
        const int e1 = (int)(y & 0x1FFFFu) - 1, t1 = (int)((y >> 17) & 0x3FFu);
        const int e2 = (int)((y >> 27) & 0x1FFFFu) - 1, t2 = (int)((y >> 44) & 0x3FFu);
        unsigned long long m1 = 0, w1 = ~0ull, w2 = ~0ull;
        ulonglong2 g2 = make_ulonglong2(0ull, 0ull);
        if (e1 >= 0) {
            m1 = __ldg(reinterpret_cast<const unsigned long long*>(seg + e1));
            w1 = ld_cg64(mrow + (uint32_t)t1 * (uint32_t)a.N);
        }
        if (e2 >= 0) {
            g2 = __ldg(seg + e2);
            w2 = ld_cg64(mrow + (uint32_t)t2 * (uint32_t)a.N);
        }
        take(t, m, w);
        if (e1 < 0) break;
        take(t1, m1, w1);
        if (e2 < 0) break;
        g = g2;
        t = t2;
        m = g.x;
        w = w2;
    }
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long v) {
    const unsigned lo = __reduce_or_sync(FULL, (unsigned)v), hi = __reduce_or_sync(FULL, (unsigned)(v >> 32));
    return (unsigned long long)hi << 32 | lo;
}

// The same fill with the walks of one warp in lockstep. A warp owns one tree
// and the 32 pixels of half an 8x8 tile (4 rows of 8: lane l is bit
// 32q + l of the tile's mark word), whose paths to the root soon merge. The
// walks advance one segment at a time, and a lane advances only while its
// segment entry is farther from the root than every lane's next entry
// (d(s, .) falls strictly along a path): a lane whose entry another lane
// will still reach waits there for it, so lanes whose paths merge take the
// shared segments in the same instructions, while lanes on separate paths
// advance side by side. The new pairs of a step are then written, tile by
// tile, per ancestor a for all its lanes at once: the column stores D[a][b]
// of the lanes form whole runs of 8 entries, and the mirror bits (row a,
// columns b) one OR of the lanes' ballot into the half of the word that
// holds the half tile. The first segment (inside the lanes' own tile) is
// taken by all lanes together. With ONE_SIDE, only D[a][b] is written (a
// pass of k_mirror completes D[b][a] afterwards).
template <bool ONE_SIDE>
__global__ void __launch_bounds__(128, FILL_G_MINB) k_fill_l(TreeArgs a, int B) {
    pdl_wait();
    pdl_trigger();
    const int nsel = *a.nsel;
    if (nsel == 0) return;
    const int lane = threadIdx.x & 31;
    // a block: one tree, four neighbouring half tiles (whose paths share
    // records and source-row entries through L1); blocks of the same half
    // tiles and all trees follow each other
    const int hg = blockIdx.x / B, j = blockIdx.x - hg * B;
    const int half = hg * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int t0 = half >> 1, q = half & 1;
    if (j >= nsel || t0 >= a.words) return;  // uniform over the warp
    const int tr = t0 / a.tiles_w, tc = t0 - tr * a.tiles_w;
    const int r = tr * 8 + q * 4 + (lane >> 3), c = tc * 8 + (lane & 7);
    const int s = a.sel[j];
    const uint32_t srow = (uint32_t)s * (uint32_t)a.N;
    bool on = r < a.H && c < a.W;
    const int b = on ? r * a.W + c : 0;
    uint32_t db = 0;
    if (on) on = b != s && __ldcg(a.cnt + b) < (uint32_t)a.N;
    if (on) {
        db = __ldg(a.D + srow + b);
        on = db != UNREACH;
    }
    if (!__any_sync(FULL, on)) return;
    unsigned long long* const mrow = a.marks + b;  // row b's word of tile t at mrow[t * N]
    const int mshift = q * 32;
    const ulonglong2* seg = a.seg + (size_t)j * a.N;
    const uint32_t* const drow = a.D + srow;  // d(s, .)
    uint32_t* const dcol = a.Dw + b;          // D[x][b] at dcol[x * N]
    uint32_t* const drowb = a.Dw + (size_t)b * a.N;
    // the mirror bits of this half tile: the low or high half of the words
    // of tile t0 (row x's at mmir[2 x])
    unsigned* const mmir = reinterpret_cast<unsigned*>(a.marks + (size_t)t0 * a.N) + q;
    // the lane's current segment: tile t, ancestor bits m, row b's mark word
    // w for t, the record's exits y and the key d(s, entry) + 1 (0: the walk
    // is over; all ones: the first segment)
    int t = t0;
    unsigned long long m = 0, w = 0, y = 0;
    uint32_t key = 0;
    if (on) {
        const ulonglong2 g = __ldg(seg + b);
        m = g.x & ~(1ull << (mshift + lane));
        y = g.y;
        w = ld_cg64(mrow + (uint32_t)t0 * (uint32_t)a.N);
        key = 0xFFFFFFFFu;
    }
    // the segment after it, fetched one step ahead
    int tn = 0;
    unsigned long long mn = 0, wn = 0, yn = 0;
    uint32_t keyn = 0;
    auto fetch = [&]() {
        const int e1 = (int)(y & 0x1FFFFu) - 1;
        keyn = 0;
        if (key != 0 && e1 >= 0) {
            tn = (int)((y >> 17) & 0x3FFu);
            const ulonglong2 g = __ldg(seg + e1);
            mn = g.x;
            yn = g.y;
            wn = ld_cg64(mrow + (uint32_t)tn * (uint32_t)a.N);
            keyn = __ldg(a.D + srow + e1) + 1;
        }
    };
    fetch();
    // every step advances at least one lane by one segment, and the keys of a
    // lane fall strictly: at most 32 N steps
    for (long long guard = 0; guard <= 32LL * a.N; ++guard) {
        if (!__any_sync(FULL, key != 0)) break;
        // a lane goes when its entry is farther from the root than every
        // lane's next entry: a lane that another one will still join waits
        // for it (the other's next entry is at or before its own), and lanes
        // on separate paths go side by side
        const uint32_t T = __reduce_max_sync(FULL, keyn);
        const bool go = key != 0 && key > T;
        unsigned long long nb = go ? m & ~w : 0ull;
        if (nb) nb &= ~atomicOr(mrow + (uint32_t)t * (uint32_t)a.N, nb);
        // the new pairs, tile by tile: the union of the lanes' new bits once
        for (unsigned gl = __ballot_sync(FULL, nb != 0); gl;) {
            const int tg = __shfl_sync(FULL, t, __ffs(gl) - 1);
            const bool in = nb != 0 && t == tg;
            gl &= ~__ballot_sync(FULL, in);
            const unsigned long long mine = in ? nb : 0ull;
            const unsigned long long U = warp_or64(mine);
            const int base = __ldg(a.tbase + tg);
            // the bits of each half of the tile (tile rows 0-3, 4-7) with
            // 32-bit operations
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned Uh = (unsigned)(U >> (32 * h));
                const unsigned mh = (unsigned)(mine >> (32 * h));
                const int bh = base + 4 * h * a.W;
                while (Uh) {
                    int ap[4], bit[4];
                    uint32_t dv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        ap[k] = -1;
                        if (Uh) {
                            bit[k] = __ffs(Uh) - 1;
                            Uh &= Uh - 1;
                            ap[k] = bh + (bit[k] >> 3) * a.W + (bit[k] & 7);
                            dv[k] = __ldg(drow + ap[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (ap[k] < 0) continue;
                        const bool has = (mh >> bit[k]) & 1u;
                        const unsigned bal = __ballot_sync(FULL, has);
                        if (has) {
                            const uint32_t val = db - dv[k];
                            if (!ONE_SIDE) __stcs(drowb + ap[k], val);
                            __stcs(dcol + (uint32_t)ap[k] * (uint32_t)a.N, val);
                        }
                        if (lane == 0) atomicOr(mmir + 2 * ap[k], bal);
                    }
                }
            }
        }
        if (go) {
            t = tn;
            m = mn;
            w = wn;
            y = yn;
            key = keyn;
            fetch();
        }
    }
}

// After a fill round that wrote only D[a][b] of its pairs (a the ancestor):
// every entry still UNREACH whose mirror is known takes the mirror's value
// (the distance is symmetric). The array starts as UNREACH, and no launch
// that writes anything but exact distances into it runs meanwhile, so a
// known entry is exact and an entry written concurrently gets the same
// value. Tiles of 64 x 64 entries in pairs (I, J), I <= J: each thread loads
// four 16-byte chunks of each tile (rows t/16 + 16q, chunk t%16), keeps them
// in registers and puts them in shared memory (row pitch 65) for the
// transposed reads; a chunk is stored back only when one of its entries
// changed. Tiles on the array's edge (or N not a multiple of 4) go entry by
// entry.
constexpr int MT = 64;

__device__ __forceinline__ bool take_mirror(uint32_t& v, uint32_t m) {
    const bool c = v == UNREACH && m != UNREACH;
    if (c) v = m;
    return c;
}

__global__ void __launch_bounds__(256) k_mirror(uint32_t* D, int N) {
    __shared__ uint32_t sa[MT * (MT + 1)], sb[MT * (MT + 1)];
    const long long T = (N + MT - 1) / MT, pairs = T * (T + 1) / 2;
    const int t = threadIdx.x, c4 = t & 15, rq = t >> 4;
    auto start = [T](long long i) { return i * T - i * (i - 1) / 2; };  // first pair of tile row i
    for (long long k = blockIdx.x; k < pairs; k += gridDim.x) {
        const double u = 2.0 * T + 1.0;
        long long I = (long long)((u - sqrt(u * u - 8.0 * (double)k)) * 0.5);
        I = I < 0 ? 0 : (I >= T ? T - 1 : I);
        while (I > 0 && start(I) > k) --I;
        while (I + 1 < T && start(I + 1) <= k) ++I;
        const long long J = I + (k - start(I));
        const int i0 = (int)(I * MT), j0 = (int)(J * MT);
        const bool diag = I == J;
        const uint32_t* mb = diag ? sa : sb;  // the mirror of tile (I, J)
        if ((N & 3) == 0 && j0 + MT <= N) {
            uint4 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rq + 16 * q;
                a[q] = __ldcs(reinterpret_cast<const uint4*>(D + (size_t)(i0 + r) * N + j0) + c4);
                if (!diag) b[q] = __ldcs(reinterpret_cast<const uint4*>(D + (size_t)(j0 + r) * N + i0) + c4);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t* x = sa + (rq + 16 * q) * (MT + 1) + 4 * c4;
                x[0] = a[q].x; x[1] = a[q].y; x[2] = a[q].z; x[3] = a[q].w;
                if (!diag) {
                    uint32_t* y = sb + (rq + 16 * q) * (MT + 1) + 4 * c4;
                    y[0] = b[q].x; y[1] = b[q].y; y[2] = b[q].z; y[3] = b[q].w;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rq + 16 * q;
                const uint32_t* m = mb + 4 * c4 * (MT + 1) + r;  // column r of the mirror, rows 4 c4 ..
                bool ch = take_mirror(a[q].x, m[0]);
                ch |= take_mirror(a[q].y, m[MT + 1]);
                ch |= take_mirror(a[q].z, m[2 * (MT + 1)]);
                ch |= take_mirror(a[q].w, m[3 * (MT + 1)]);
                if (ch) *(reinterpret_cast<uint4*>(D + (size_t)(i0 + r) * N + j0) + c4) = a[q];
                if (!diag) {
                    const uint32_t* n = sa + 4 * c4 * (MT + 1) + r;
                    bool cb = take_mirror(b[q].x, n[0]);
                    cb |= take_mirror(b[q].y, n[MT + 1]);
                    cb |= take_mirror(b[q].z, n[2 * (MT + 1)]);
                    cb |= take_mirror(b[q].w, n[3 * (MT + 1)]);
                    if (cb) *(reinterpret_cast<uint4*>(D + (size_t)(j0 + r) * N + i0) + c4) = b[q];
                }
            }
            __syncthreads();
            continue;
        }
        const int tx = t & (MT - 1), ty = t / MT;
        for (int r = ty; r < MT; r += 256 / MT) {
            const int i = i0 + r, j = j0 + tx, i2 = j0 + r, j2 = i0 + tx;
            sa[r * (MT + 1) + tx] = (i < N && j < N) ? __ldcs(D + (size_t)i * N + j) : UNREACH;
            sb[r * (MT + 1) + tx] = (!diag && i2 < N && j2 < N) ? __ldcs(D + (size_t)i2 * N + j2) : UNREACH;
        }
        __syncthreads();
        for (int r = ty; r < MT; r += 256 / MT) {
            const int i = i0 + r, j = j0 + tx, i2 = j0 + r, j2 = i0 + tx;
            uint32_t v = sa[r * (MT + 1) + tx];
            if (i < N && j < N && take_mirror(v, mb[tx * (MT + 1) + r])) D[(size_t)i * N + j] = v;
            uint32_t w = sb[r * (MT + 1) + tx];
            if (!diag && i2 < N && j2 < N && take_mirror(w, sa[tx * (MT + 1) + r])) D[(size_t)i2 * N + j2] = w;
        }
        __syncthreads();
    }
}

// Fill counts of the rows still open: cnt(x) = cnt at the start + the
// number of marked pairs of row x (both bits of a pair are set, so row x
// holds every filled pair {x, y}). A block takes 32 consecutive rows, its
// eight warps an eighth of the tiles each: a warp reads the same tile's
// words of the 32 rows at once. Rows already filled (cnt = N) cannot
// change. Recounting every open row costs one streaming
// read of its marks, where flagging the rows that changed cost the fill a
// store per new pair. The increments are summed into S_NEW, which thus
// counts every new pair twice.
__global__ void k_recount(TreeArgs a) {
    __shared__ unsigned long long s_sum;
    pdl_wait();
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    __shared__ unsigned s_part[8][32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const bool open = x < a.N && __ldcg(a.cnt + x) < (uint32_t)a.N;
    unsigned c = 0;
    if (__syncthreads_or(open)) {
        if (open) {
            const unsigned long long* col = a.marks + x;
#pragma unroll 4
            for (int w = wp; w < a.words; w += 8) c += __popcll(__ldcg(col + (size_t)w * a.N));
        }
        s_part[wp][lane] = c;
        __syncthreads();
        if (wp == 0 && open) {
            unsigned t = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += s_part[k][lane];
            const uint32_t nc = a.cnt_base[x] + t;
            atomicAdd(&s_sum, (unsigned long long)(nc - a.cnt[x]));
            a.cnt[x] = nc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(a.stats + S_NEW, s_sum);
}

}  // namespace

// cudaLaunchKernelEx with an optional cluster size and the programmatic
// dependent launch attribute.
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, bool pdl,
                      int cluster, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    int n = 0;
    if (cluster > 1) {
        at[n].id = cudaLaunchAttributeClusterDimension;
        at[n].val.clusterDim.x = cluster;
        at[n].val.clusterDim.y = 1;
        at[n].val.clusterDim.z = 1;
        ++n;
    }
    if (pdl) {
        at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_recount(const TreeArgs& a, cudaStream_t st, bool pdl) {
    return launch_ex(k_recount, (a.N + 31) / 32, 256, 0, st, pdl, 1, a);
}

cudaError_t launch_tree(const TreeArgs& a, int B, cudaStream_t st, bool pdl) {
    if (a.N <= 16384 && a.dep_exit && a.H >= 16) {
        // several blocks (one cluster) per tree: four strips when they are
        // 16 rows or more, else two
        if (a.H >= 64) {
            const TreeCLayout L(a.H, a.W, 4, level_bytes(a.kind));
            static std::atomic<unsigned long long> attr4{0};
            once_per_device(attr4, [] {
                cudaFuncSetAttribute(k_treeC<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            });
            return launch_ex(k_treeC<4>, 4 * B, 1024, L.bytes(), st, pdl, 4, a);
        }
        const TreeCLayout L(a.H, a.W, 2, level_bytes(a.kind));
        static std::atomic<unsigned long long> attr2{0};
        once_per_device(attr2, [] {
            cudaFuncSetAttribute(k_treeC<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        return launch_ex(k_treeC<2>, 2 * B, 1024, L.bytes(), st, pdl, 2, a);
    }
    if (a.N <= 16384) {
        static std::atomic<unsigned long long> attr{0};
        once_per_device(attr, [] {
            cudaFuncSetAttribute(k_tree<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 12);
        });
        // five 16-bit arrays and the image
        return launch_ex(k_tree<true>, B, 1024, (size_t)a.N * (10 + level_bytes(a.kind)), st, pdl, 1, a);
    }
    if (a.H >= 64) {
        // N > 16384 (so H > 64): eight strips of whole tiles, when a cluster
        // of eight such blocks can be resident at all
        const TreeWLayout L(a.H, a.W, 8, level_bytes(a.kind));
        static std::atomic<unsigned long long> attr8{0};
        once_per_device(attr8, [] {
            cudaFuncSetAttribute(k_treeW<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        if (L.bytes() <= 200 * 1024) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(8);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = L.bytes();
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 8;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, k_treeW<8>, &cfg) == cudaSuccess && clusters > 0)
                return launch_ex(k_treeW<8>, 8 * B, 1024, L.bytes(), st, pdl, 8, a);
            cudaGetLastError();
        }
    }
    return launch_ex(k_tree<false>, B, 1024, 0, st, pdl, 1, a);
}

cudaError_t launch_depths(const TreeArgs& a, int B, cudaStream_t st) {
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_depths, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8);
    });
    k_depths<<<B, 1024, (size_t)a.N * 8, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mirror(uint32_t* D, int N, cudaStream_t st) {
    const long long T = (N + MT - 1) / MT, pairs = T * (T + 1) / 2;
    const long long grid = pairs < 152 * 4 ? pairs : 152 * 4;
    k_mirror<<<(unsigned)grid, 256, 0, st>>>(D, N);
    return cudaGetLastError();
}

cudaError_t launch_fill(const TreeArgs& a, int B, cudaStream_t st, bool pdl) {
    if (a.rows_per_block < 0) {
        // walks in lockstep: one warp per half tile and tree
        const long long groups = (2LL * a.words + 3) / 4;
        if (a.one_side) return launch_ex(k_fill_l<true>, (int)(groups * B), 128, 0, st, pdl, 1, a, B);
        return launch_ex(k_fill_l<false>, (int)(groups * B), 128, 0, st, pdl, 1, a, B);
    }
    if (a.rows_per_block == 0) {
        // marks claimed in global memory: one warp per 8 rows x 4 trees
        const int quads = (B + 3) / 4;
        const long long warps = (long long)((a.N + 7) / 8) * quads;
        return launch_ex(k_fill_g, (int)((warps + 3) / 4), 128, 0, st, pdl, 1, a, quads);
    }
    // mark rows, then one "changed" byte per row word
    const size_t smem = fill_smem_bytes(a.rows_per_block, a.words);
    static std::atomic<unsigned long long> attr_set{0};
    once_per_device(attr_set, [] {
        cudaFuncSetAttribute(k_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    const int grid = (a.N + a.rows_per_block - 1) / a.rows_per_block;
    return launch_ex(k_fill, grid, 256, smem, st, pdl, 1, a);
}

}  // namespace gapsp
