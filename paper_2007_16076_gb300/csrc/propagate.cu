// Kernel (a): geodesic propagation on the image graph.
//
// Computes d(s, .) = min over paths of the summed edge weights (Sec. 2, eqs.
// "temps" and "distance"), the "geodesic time function" of Soille used by
// the paper with a 3x3 neighbourhood (Sec. 3). Weights are w(p,q) = f(p) +
// f(q) + 1 (grey) or 2 between free pixels (mask).
//
// One warp owns one source (or one multi-source seed set) and drives its map
// to the exact fixpoint with directional sweeps. A sweep visits the lines of
// the image in order (rows top-down, rows bottom-up, columns left-right,
// columns right-left). For each line it
//   1. relaxes every pixel from the already-final previous line (the 3
//      neighbours above for 8-connectivity, 1 for 4), then
//   2. closes the line in both directions at once: with P the prefix sum of
//      the line's edge weights, the best value reachable along the line is
//      min_c' v(c') + |P(c) - P(c')|, i.e. a prefix-min of v - P and a
//      suffix-min of v + P (warp shuffles; skipped when a neighbour test
//      shows the line is already closed).
// A line of up to 32*VPL pixels lives in registers, lane j holding pixels
// j, j+32, ... so that both row and column lines load without shared-memory
// bank conflicts. All weights are >= 1 and integral, so the fixpoint is
// unique and equal to the Dijkstra distances whatever the sweep schedule.
// The warp stops when two sweeps that together test every edge direction
// (down+up or right+left, or any three in a row) change nothing, and gives
// up with a status bit after max_sweeps.
#include "common.cuh"
#include "internal.h"

namespace gapsp {

namespace {

// Where a warp keeps its distance map: shared memory (row pitch odd, so both
// row lines and column lines hit 32 distinct banks), or global memory for
// images too large for shared memory.
struct SmemMap {
    int* base;
    int pitch;
    __device__ __forceinline__ int ld(int e_r, int e_c) const { return base[e_r * pitch + e_c]; }
    __device__ __forceinline__ void st(int e_r, int e_c, int v) const { base[e_r * pitch + e_c] = v; }
};
struct GlobMap {
    int* base;
    int pitch;
    __device__ __forceinline__ int ld(int e_r, int e_c) const { return ld_cg(base + e_r * pitch + e_c); }
    __device__ __forceinline__ void st(int e_r, int e_c, int v) const { base[e_r * pitch + e_c] = v; }
};

template <int VPL>
struct Line {
    int o[VPL];  // value before this sweep
    int f[VPL];  // grey level (grey) or free flag (mask)
    int p[VPL];  // line prefix of edge weights
};

template <int KIND, int VPL, bool ROWS, class Map>
__device__ __forceinline__ void load_line(const PropArgs& a, const Map& map, int src, bool first,
                                          int l, int len, int lane, Line<VPL>& L) {
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        int pos = lane + 32 * k;
        if (pos < len) {
            int e = ROWS ? l * a.W + pos : pos * a.W + l;
            if (first) {
                bool seed = a.seed_flags ? (a.seed_flags[e] != 0) : (e == src);
                L.o[k] = seed ? 0 : PINF;
            } else {
                L.o[k] = ROWS ? map.ld(l, pos) : map.ld(pos, l);
            }
            L.f[k] = __ldg(a.f + e);
            if (KIND == 0) {
                const int* P = ROWS ? a.Prow : a.Pcol;
                L.p[k] = __ldg(P + l * len + pos);
            } else {
                L.p[k] = 2 * pos;
            }
        } else {
            L.o[k] = PINF;
            L.f[k] = 0;
            L.p[k] = 0;
        }
    }
}

// Value of the pixel one position before (UP) or after (!UP) each held pixel,
// taken from another lane; `edge` fills the ends of the line.
template <int VPL, bool UP>
__device__ __forceinline__ void rotate(const int (&v)[VPL], int (&out)[VPL], int lane, int edge) {
    int r[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) r[k] = __shfl_sync(FULL, v[k], UP ? (lane + 31) & 31 : (lane + 1) & 31);
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        if (UP) out[k] = lane == 0 ? (k > 0 ? r[k - 1] : edge) : r[k];
        else out[k] = lane == 31 ? (k + 1 < VPL ? r[k + 1] : edge) : r[k];
    }
}

template <int CONN, int KIND, int VPL, bool ROWS, class Map>
__device__ bool sweep(const PropArgs& a, const Map& map, int src, bool first, int dir, int lane) {
    const int nlines = ROWS ? a.H : a.W;
    const int len = ROWS ? a.W : a.H;
    int l = dir > 0 ? 0 : nlines - 1;
    Line<VPL> cur, nxt;
    load_line<KIND, VPL, ROWS, Map>(a, map, src, first, l, len, lane, cur);
    int dp[VPL], fp[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) { dp[k] = PINF; fp[k] = 0; }
    bool changed = false;
    for (int i = 0; i < nlines; ++i, l += dir) {
        if (i + 1 < nlines) load_line<KIND, VPL, ROWS, Map>(a, map, src, first, l + dir, len, lane, nxt);
        // 1. relax from the previous line
        int dl[VPL], dr[VPL], fl[VPL], fr[VPL];
        if (CONN == 8) {
            rotate<VPL, true>(dp, dl, lane, PINF);
            rotate<VPL, false>(dp, dr, lane, PINF);
            if (KIND == 0) {
                rotate<VPL, true>(fp, fl, lane, 0);
                rotate<VPL, false>(fp, fr, lane, 0);
            }
        }
        int v[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            int best = cur.o[k];
            if (KIND == 0) {
                int fc1 = cur.f[k] + 1;
                best = min(best, dp[k] + fp[k] + fc1);
                if (CONN == 8) {
                    best = min(best, dl[k] + fl[k] + fc1);
                    best = min(best, dr[k] + fr[k] + fc1);
                }
            } else {
                best = min(best, dp[k] + 2);
                if (CONN == 8) best = min(best, min(dl[k], dr[k]) + 2);
                if (!cur.f[k]) best = PINF;  // obstacles keep no distance
            }
            v[k] = (lane + 32 * k < len) ? best : PINF;
        }
        // 2. close the line: prefix-min of v - P and suffix-min of v + P
        int x[VPL], y[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) { x[k] = v[k] - cur.p[k]; y[k] = v[k] + cur.p[k]; }
        unsigned ob[VPL];
        if (KIND == 1) {
#pragma unroll
            for (int k = 0; k < VPL; ++k) ob[k] = __ballot_sync(FULL, !(lane + 32 * k < len && cur.f[k]));
        }
        bool need = false;
        {
            int xl[VPL], yr[VPL];
            rotate<VPL, true>(x, xl, lane, PINF);
            rotate<VPL, false>(y, yr, lane, PINF);
#pragma unroll
            for (int k = 0; k < VPL; ++k)
                need |= (lane + 32 * k < len) && (KIND == 0 || cur.f[k]) && (xl[k] < x[k] || yr[k] < y[k]);
        }
        int d[VPL];
        if (__any_sync(FULL, need)) {
            int sx[VPL], sy[VPL];
#pragma unroll
            for (int k = 0; k < VPL; ++k) { sx[k] = x[k]; sy[k] = y[k]; }
#pragma unroll
            for (int delta = 1; delta < 32; delta <<= 1) {
#pragma unroll
                for (int k = 0; k < VPL; ++k) {
                    int t = __shfl_up_sync(FULL, sx[k], delta);
                    int u = __shfl_down_sync(FULL, sy[k], delta);
                    bool okx = lane >= delta, oky = lane + delta < 32;
                    if (KIND == 1) {
                        // combine only inside a run of free pixels
                        unsigned m = (1u << delta) - 1u;
                        okx = okx && (((ob[k] >> (okx ? lane - delta : 0)) & m) == 0u);
                        oky = oky && (((ob[k] >> (oky ? lane + 1 : 0)) & m) == 0u);
                    }
                    if (okx) sx[k] = min(sx[k], t);
                    if (oky) sy[k] = min(sy[k], u);
                }
            }
            // chain the 32-pixel chunks
            int carry = PINF;
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                bool ok = true;
                if (KIND == 1)
                    ok = k > 0 && !((ob[k - 1] >> 31) & 1u) && ((ob[k] & ((1u << lane) - 1u)) == 0u);
                if (ok) sx[k] = min(sx[k], carry);
                carry = __shfl_sync(FULL, sx[k], 31);
            }
            carry = PINF;
#pragma unroll
            for (int k = VPL - 1; k >= 0; --k) {
                bool ok = true;
                if (KIND == 1) {
                    unsigned after = lane == 31 ? 0u : (ob[k] >> (lane + 1));
                    ok = k + 1 < VPL && !(ob[k + 1] & 1u) && after == 0u;
                }
                if (ok) sy[k] = min(sy[k], carry);
                carry = __shfl_sync(FULL, sy[k], 0);
            }
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                int r = min(v[k], min(sx[k] + cur.p[k], sy[k] - cur.p[k]));
                if (KIND == 1 && !cur.f[k]) r = PINF;
                d[k] = (lane + 32 * k < len) ? r : PINF;
            }
        } else {
#pragma unroll
            for (int k = 0; k < VPL; ++k) d[k] = v[k];
        }
        // store what changed (everything on the first sweep)
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            int pos = lane + 32 * k;
            if (pos < len) {
                bool ch = d[k] != cur.o[k];
                changed |= ch;
                if (ch || first) {
                    if (ROWS) map.st(l, pos, d[k]);
                    else map.st(pos, l, d[k]);
                }
            }
            dp[k] = d[k];
            fp[k] = cur.f[k];
        }
        if (i + 1 < nlines) cur = nxt;
    }
    return __any_sync(FULL, changed);
}

// Sweeps until the fixpoint; returns the number of sweeps.
template <int CONN, int KIND, int VPL, class Map>
__device__ int drive(const PropArgs& a, const Map& map, int src, int lane) {
    int nsweep = 0, run = 0;
    for (;;) {
        const bool first = nsweep == 0;
        bool ch;
        switch (nsweep & 3) {
            case 0: ch = sweep<CONN, KIND, VPL, true>(a, map, src, first, +1, lane); break;
            case 1: ch = sweep<CONN, KIND, VPL, true>(a, map, src, first, -1, lane); break;
            case 2: ch = sweep<CONN, KIND, VPL, false>(a, map, src, first, +1, lane); break;
            default: ch = sweep<CONN, KIND, VPL, false>(a, map, src, first, -1, lane); break;
        }
        __syncwarp();
        run = (ch || first) ? 0 : run + 1;
        ++nsweep;
        // Two unchanged sweeps of an opposite pair (down+up, right+left) test
        // every edge; for 4-connectivity any two distinct sweeps do. Three in
        // a row always contain an opposite pair.
        const bool done = CONN == 4 ? run >= 2 : (run >= 3 || (run >= 2 && ((nsweep - 1) & 1)));
        if (done) break;
        if (nsweep >= a.max_sweeps) {
            if (lane == 0) atomicOr(a.status, ST_NOT_CONVERGED);
            break;
        }
    }
    return nsweep;
}

__device__ __forceinline__ int finish(const PropArgs& a, int v) {
    return (a.convert && v >= PINF) ? (int)UNREACH : v;
}

// Map in shared memory: one warp per block.
template <int CONN, int KIND, int VPL>
__global__ void __launch_bounds__(32) k_propagate_smem(PropArgs a, int pitch) {
    extern __shared__ int smap[];
    const int lane = threadIdx.x;
    const int j = blockIdx.x;
    const int njobs = a.njobs_dev ? *a.njobs_dev : a.njobs;
    if (j >= njobs) return;
    const int src = a.sources ? a.sources[j] : -1;
    int* out = a.map_base + (size_t)(a.map_row ? a.map_row[j] : j) * (size_t)a.N;
    const SmemMap map{smap, pitch};
    const int ns = drive<CONN, KIND, VPL>(a, map, src, lane);
    if (lane == 0 && a.sweeps) atomicAdd(a.sweeps, (unsigned long long)ns);
    // coalesced store of the finished row, four pixels per lane per step
    if ((a.N & 3) == 0 && (a.W & 3) == 0) {
        int4* o4 = reinterpret_cast<int4*>(out);
        for (int q = lane; q < a.N / 4; q += 32) {
            const int p = 4 * q, r = p / a.W, c = p - r * a.W;
            const int* m = smap + r * pitch + c;
            o4[q] = make_int4(finish(a, m[0]), finish(a, m[1]), finish(a, m[2]), finish(a, m[3]));
        }
    } else {
        for (int p = lane; p < a.N; p += 32) {
            const int r = p / a.W, c = p - r * a.W;
            out[p] = finish(a, smap[r * pitch + c]);
        }
    }
    __syncwarp();
    if (lane == 0 && a.convert && src >= 0 && KIND == 1 && !a.f[src]) out[src] = 0;
}

// Map in global memory (images too large for shared memory).
template <int CONN, int KIND, int VPL>
__global__ void k_propagate_glob(PropArgs a) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int njobs = a.njobs_dev ? *a.njobs_dev : a.njobs;
    if (j >= njobs) return;
    const int src = a.sources ? a.sources[j] : -1;
    int* map = a.map_base + (size_t)(a.map_row ? a.map_row[j] : j) * (size_t)a.N;
    const GlobMap gm{map, a.W};
    const int ns = drive<CONN, KIND, VPL>(a, gm, src, lane);
    if (lane == 0 && a.sweeps) atomicAdd(a.sweeps, (unsigned long long)ns);
    if (a.convert) {
        for (int p = lane; p < a.N; p += 32) {
            int v = ld_cg(map + p);
            if (v >= PINF) map[p] = (int)UNREACH;
        }
        __syncwarp();
        if (lane == 0 && src >= 0 && KIND == 1 && !a.f[src]) map[src] = 0;
    }
}

constexpr int SMEM_MAP_LIMIT = 200 * 1024;

int smem_pitch(int W) { return W | 1; }

template <int CONN, int KIND, int VPL>
cudaError_t launch_one(const PropArgs& a, int grid, int wpb, cudaStream_t st) {
    const int pitch = smem_pitch(a.W);
    const size_t smem = (size_t)a.H * pitch * sizeof(int);
    if (smem <= (size_t)SMEM_MAP_LIMIT) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_propagate_smem<CONN, KIND, VPL>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_MAP_LIMIT);
            attr = true;
        }
        // one warp (one job) per block
        const int jobs = grid * wpb;
        k_propagate_smem<CONN, KIND, VPL><<<jobs, 32, smem, st>>>(a, pitch);
    } else {
        k_propagate_glob<CONN, KIND, VPL><<<grid, 32 * wpb, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int CONN, int KIND>
cudaError_t launch_vpl(const PropArgs& a, int vpl, int grid, int wpb, cudaStream_t st) {
    switch (vpl) {
        case 1: return launch_one<CONN, KIND, 1>(a, grid, wpb, st);
        case 2: return launch_one<CONN, KIND, 2>(a, grid, wpb, st);
        case 4: return launch_one<CONN, KIND, 4>(a, grid, wpb, st);
        case 8: return launch_one<CONN, KIND, 8>(a, grid, wpb, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int prop_vpl(int side) {
    if (side <= 32) return 1;
    if (side <= 64) return 2;
    if (side <= 128) return 4;
    if (side <= 256) return 8;
    return -1;
}

cudaError_t launch_propagate(const PropArgs& a, int conn, int kind, int grid, int wpb, cudaStream_t st) {
    int vpl = prop_vpl(a.H > a.W ? a.H : a.W);
    if (grid <= 0) return cudaSuccess;
    if (conn == 8) return kind == 0 ? launch_vpl<8, 0>(a, vpl, grid, wpb, st) : launch_vpl<8, 1>(a, vpl, grid, wpb, st);
    return kind == 0 ? launch_vpl<4, 0>(a, vpl, grid, wpb, st) : launch_vpl<4, 1>(a, vpl, grid, wpb, st);
}

// ---------------------------------------------------------------------------
// Per-image set-up: line prefixes of the edge weights and boundary flags.
// ---------------------------------------------------------------------------

namespace {

// One thread per line: Prow[r][c] = sum_{k<c} w((r,k),(r,k+1)) (grey only).
__global__ void k_prefix(ImagePrep p) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < p.H) {
        int r = t, acc = 0;
        for (int c = 0; c < p.W; ++c) {
            p.Prow[r * p.W + c] = acc;
            if (c + 1 < p.W) acc += p.f[r * p.W + c] + p.f[r * p.W + c + 1] + 1;
        }
    } else if (t < p.H + p.W) {
        int c = t - p.H, acc = 0;
        for (int r = 0; r < p.H; ++r) {
            p.Pcol[c * p.H + r] = acc;
            if (r + 1 < p.H) acc += p.f[r * p.W + c] + p.f[(r + 1) * p.W + c] + 1;
        }
    }
}

// Boundary vertices: free pixels with fewer free neighbours than the
// connectivity (the image edges on a full grid; Sec. 3.3 and Sec. 5).
__global__ void k_boundary(ImagePrep p) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int N = p.H * p.W;
    if (q >= N) return;
    int r = q / p.W, c = q - r * p.W;
    bool fr = p.kind == 0 || p.f[q];
    int n = 0;
    for (int dr = -1; dr <= 1; ++dr)
        for (int dc = -1; dc <= 1; ++dc) {
            if (!dr && !dc) continue;
            if (p.conn == 4 && dr && dc) continue;
            int rr = r + dr, cc = c + dc;
            if (rr < 0 || rr >= p.H || cc < 0 || cc >= p.W) continue;
            if (p.kind == 1 && !p.f[rr * p.W + cc]) continue;
            ++n;
        }
    p.bound[q] = (fr && n < p.conn) ? 1 : 0;
}

__global__ void k_unreach(uint32_t* rows, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride)
        if ((int)rows[i] >= PINF) rows[i] = UNREACH;
}

}  // namespace

cudaError_t launch_image_prep(const ImagePrep& p, cudaStream_t st) {
    int lines = p.H + p.W;
    if (p.kind == 0) k_prefix<<<(lines + 127) / 128, 128, 0, st>>>(p);
    int N = p.H * p.W;
    k_boundary<<<(N + 255) / 256, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_unreach_convert(uint32_t* rows, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_unreach<<<1216, 256, 0, st>>>(rows, n);
    return cudaGetLastError();
}

}  // namespace gapsp
