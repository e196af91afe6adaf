// Kernel (a): geodesic propagation on the image graph.
//
// Computes d(s, .) = min over paths of the summed edge weights (Sec. 2, eqs.
// "temps" and "distance"), the "geodesic time function" of Soille that the
// paper uses with a 3x3 neighbourhood (Sec. 3). Weights are w(p,q) = f(p) +
// f(q) + 1 (grey) or 2 between free pixels (mask).
//
// One block of four warps owns one source (or one multi-source seed set).
// Its distance map sits in shared memory (global memory for images too
// large), initialised to 0 at the seeds and "unreached" elsewhere. The four
// warps sweep the map concurrently, each in its own direction: rows
// top-down, rows bottom-up, columns left-right, columns right-left. For
// each line a warp
//   1. relaxes every pixel from the previous line it just finished (the
//      three neighbours behind it for 8-connectivity, one for 4), then
//   2. closes the line in both directions: with P the prefix sum of the
//      line's edge weights, the best value along the line is
//      min_c' v(c') + |P(c) - P(c')|, a prefix-min of v - P and a suffix-min
//      of v + P. Lane j holds pixels VPL*j .. VPL*j+VPL-1, so the scans run
//      inside the lane and need warp shuffles only when a boundary test
//      shows that a value must cross from one lane to another,
// and lowers the map with atomic minima. Every stored value is the cost of
// a real path, so values only decrease towards the distances; the edge
// weights are positive integers, so the fixpoint is unique and any schedule
// reaches it. The block stops after a round (one sweep per warp) in which
// no warp lowered anything: the map was then constant while every edge
// direction was tested. Rounds are capped; hitting the cap sets a status
// bit instead of looping on.
#include "common.cuh"
#include "internal.h"

namespace gapsp {

namespace {

constexpr int PWARPS = 4;                 // one warp per sweep direction
constexpr int BIGX = PINF;                // identity of the prefix-min of v - P
constexpr int BIGY = PINF + (1 << 18);    // identity of the suffix-min of v + P

struct SmemMap {
    int* base;
    int pitch;
    __device__ __forceinline__ int ld(int r, int c) const {
        return *((volatile const int*)(base + r * pitch + c));
    }
    __device__ __forceinline__ void lower(int r, int c, int v) const { atomicMin(base + r * pitch + c, v); }
};

struct GlobMap {
    int* base;
    int pitch;
    __device__ __forceinline__ int ld(int r, int c) const { return ld_cg(base + r * pitch + c); }
    __device__ __forceinline__ void lower(int r, int c, int v) const { atomicMin(base + r * pitch + c, v); }
};

template <int VPL>
struct Line {
    int o[VPL];  // map value when loaded
    int f[VPL];  // grey level (grey) or free flag (mask)
    int p[VPL];  // prefix of the line's edge weights
};

template <int KIND, int VPL, bool ROWS, class Map>
__device__ __forceinline__ void load_line(const PropArgs& a, const Map& map, int l, int len, int lane,
                                          Line<VPL>& L) {
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int pos = VPL * lane + k;
        if (pos < len) {
            const int e = ROWS ? l * a.W + pos : pos * a.W + l;
            L.o[k] = ROWS ? map.ld(l, pos) : map.ld(pos, l);
            L.f[k] = __ldg(a.f + e);
            L.p[k] = KIND == 0 ? __ldg((ROWS ? a.Prow : a.Pcol) + l * len + pos) : 2 * pos;
        } else {
            L.o[k] = PINF;
            L.f[k] = 0;
            L.p[k] = 0;
        }
    }
}

// One sweep over all lines in one direction; true if this warp lowered
// (or may have lowered) some value.
template <int CONN, int KIND, int VPL, bool ROWS, class Map>
__device__ bool sweep(const PropArgs& a, const Map& map, int dir, int lane) {
    const int nlines = ROWS ? a.H : a.W;
    const int len = ROWS ? a.W : a.H;
    int l = dir > 0 ? 0 : nlines - 1;
    Line<VPL> cur, nxt;
    load_line<KIND, VPL, ROWS, Map>(a, map, l, len, lane, cur);
    int dp[VPL], fp[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) { dp[k] = PINF; fp[k] = 0; }
    bool changed = false;
    for (int i = 0; i < nlines; ++i, l += dir) {
        if (i + 1 < nlines) load_line<KIND, VPL, ROWS, Map>(a, map, l + dir, len, lane, nxt);
        bool valid[VPL], freep[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            valid[k] = VPL * lane + k < len;
            freep[k] = valid[k] && (KIND == 0 || cur.f[k] != 0);
        }
        // 1. relax from the previous line
        int dl0 = PINF, dr0 = PINF, fl0 = 0, fr0 = 0;
        if (CONN == 8) {
            dl0 = __shfl_up_sync(FULL, dp[VPL - 1], 1);
            dr0 = __shfl_down_sync(FULL, dp[0], 1);
            if (lane == 0) dl0 = PINF;
            if (lane == 31) dr0 = PINF;
            if (KIND == 0) {
                fl0 = __shfl_up_sync(FULL, fp[VPL - 1], 1);
                fr0 = __shfl_down_sync(FULL, fp[0], 1);
            }
        }
        int v[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            int best = cur.o[k];
            if (KIND == 0) {
                const int fc1 = cur.f[k] + 1;
                best = min(best, dp[k] + fp[k] + fc1);
                if (CONN == 8) {
                    const int dl = k > 0 ? dp[k - 1] : dl0, fl = k > 0 ? fp[k - 1] : fl0;
                    const int dr = k + 1 < VPL ? dp[k + 1] : dr0, fr = k + 1 < VPL ? fp[k + 1] : fr0;
                    best = min(best, min(dl + fl, dr + fr) + fc1);
                }
            } else {
                best = min(best, dp[k] + 2);
                if (CONN == 8) {
                    const int dl = k > 0 ? dp[k - 1] : dl0;
                    const int dr = k + 1 < VPL ? dp[k + 1] : dr0;
                    best = min(best, min(dl, dr) + 2);
                }
            }
            v[k] = freep[k] ? best : PINF;
        }
        // 2. close the line inside each lane
        int sx[VPL], sy[VPL], d[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int x = freep[k] ? v[k] - cur.p[k] : BIGX;
            sx[k] = (KIND == 1 && !freep[k]) ? BIGX : min(k > 0 ? sx[k - 1] : BIGX, x);
        }
#pragma unroll
        for (int k = VPL - 1; k >= 0; --k) {
            const int y = freep[k] ? v[k] + cur.p[k] : BIGY;
            sy[k] = (KIND == 1 && !freep[k]) ? BIGY : min(k + 1 < VPL ? sy[k + 1] : BIGY, y);
        }
#pragma unroll
        for (int k = 0; k < VPL; ++k)
            d[k] = freep[k] ? min(v[k], min(sx[k] + cur.p[k], sy[k] - cur.p[k])) : PINF;
        // does a value have to cross a lane boundary?
        const int xl = freep[VPL - 1] ? d[VPL - 1] - cur.p[VPL - 1] : BIGX;
        const int yf = freep[0] ? d[0] + cur.p[0] : BIGY;
        const int xl_left = __shfl_up_sync(FULL, xl, 1);
        const int yf_right = __shfl_down_sync(FULL, yf, 1);
        const bool need = (lane > 0 && freep[0] && xl_left < d[0] - cur.p[0]) ||
                          (lane < 31 && freep[VPL - 1] && yf_right < d[VPL - 1] + cur.p[VPL - 1]);
        if (__any_sync(FULL, need)) {
            // exclusive prefix-min of the lane totals of v - P (suffix-min of
            // v + P); on a mask, runs of free pixels are separate segments
            int tx = sx[VPL - 1], ty = sy[0];
            bool hx = false, hy = false;  // lane holds a segment start (mask)
            int first_ob = VPL, last_ob = -1;
            if (KIND == 1) {
#pragma unroll
                for (int k = VPL - 1; k >= 0; --k) if (!freep[k]) first_ob = k;
#pragma unroll
                for (int k = 0; k < VPL; ++k) if (!freep[k]) last_ob = k;
                hx = hy = first_ob < VPL;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int tx2 = __shfl_up_sync(FULL, tx, o);
                const int ty2 = __shfl_down_sync(FULL, ty, o);
                const bool hx2 = __shfl_up_sync(FULL, hx, o);
                const bool hy2 = __shfl_down_sync(FULL, hy, o);
                if (lane >= o && !hx) { tx = min(tx, tx2); hx = hx2; }
                if (lane + o < 32 && !hy) { ty = min(ty, ty2); hy = hy2; }
            }
            int ex = __shfl_up_sync(FULL, tx, 1);
            int ey = __shfl_down_sync(FULL, ty, 1);
            if (lane == 0) ex = BIGX;
            if (lane == 31) ey = BIGY;
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                if (!freep[k]) continue;
                const int px = (KIND == 1 && k > first_ob) ? sx[k] : min(ex, sx[k]);
                const int py = (KIND == 1 && k < last_ob) ? sy[k] : min(ey, sy[k]);
                d[k] = min(v[k], min(px + cur.p[k], py - cur.p[k]));
            }
        }
        // lower the map where this line improved
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            if (freep[k] && d[k] < cur.o[k]) {
                changed = true;
                const int pos = VPL * lane + k;
                if (ROWS) map.lower(l, pos, d[k]);
                else map.lower(pos, l, d[k]);
            }
            dp[k] = d[k];
            fp[k] = cur.f[k];
        }
        if (i + 1 < nlines) cur = nxt;
    }
    return __any_sync(FULL, changed);
}

template <int CONN, int KIND, int VPL, class Map>
__device__ void run_block(const PropArgs& a, const Map& map, int* s_flag, int* s_rounds) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int round = 0;
    for (;;) {
        bool ch;
        switch (warp) {
            case 0: ch = sweep<CONN, KIND, VPL, true, Map>(a, map, +1, lane); break;
            case 1: ch = sweep<CONN, KIND, VPL, true, Map>(a, map, -1, lane); break;
            case 2: ch = sweep<CONN, KIND, VPL, false, Map>(a, map, +1, lane); break;
            default: ch = sweep<CONN, KIND, VPL, false, Map>(a, map, -1, lane); break;
        }
        if (lane == 0 && ch) s_flag[round & 1] = 1;
        __syncthreads();
        const bool any = s_flag[round & 1] != 0;
        if (threadIdx.x == 0) s_flag[(round + 1) & 1] = 0;
        ++round;
        if (!any) break;
        if (round * PWARPS >= a.max_sweeps) {
            if (threadIdx.x == 0) atomicOr(a.status, ST_NOT_CONVERGED);
            break;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *s_rounds = round;
}

__device__ __forceinline__ int finish(const PropArgs& a, int v) {
    return (a.convert && v >= PINF) ? (int)UNREACH : v;
}

__device__ __forceinline__ bool is_seed(const PropArgs& a, int src, int p) {
    return a.seed_flags ? a.seed_flags[p] != 0 : p == src;
}

// Map in shared memory; one block of PWARPS warps per job.
template <int CONN, int KIND, int VPL>
__global__ void __launch_bounds__(32 * PWARPS) k_propagate_smem(PropArgs a, int pitch) {
    extern __shared__ int smap[];
    __shared__ int s_flag[2], s_rounds;
    const int j = blockIdx.x;
    const int njobs = a.njobs_dev ? *a.njobs_dev : a.njobs;
    if (j >= njobs) return;
    const int src = a.sources ? a.sources[j] : -1;
    int* out = a.map_base + (size_t)(a.map_row ? a.map_row[j] : j) * (size_t)a.N;
    for (int p = threadIdx.x; p < a.N; p += blockDim.x) {
        const int r = p / a.W, c = p - r * a.W;
        smap[r * pitch + c] = is_seed(a, src, p) ? 0 : PINF;
    }
    if (threadIdx.x == 0) { s_flag[0] = 0; s_flag[1] = 0; }
    __syncthreads();
    const SmemMap map{smap, pitch};
    run_block<CONN, KIND, VPL>(a, map, s_flag, &s_rounds);
    __syncthreads();
    if (threadIdx.x == 0 && a.sweeps) atomicAdd(a.sweeps, (unsigned long long)s_rounds * PWARPS);
    // finished row: coalesced 128-bit stores
    if ((a.N & 3) == 0 && (a.W & 3) == 0) {
        int4* o4 = reinterpret_cast<int4*>(out);
        for (int q = threadIdx.x; q < a.N / 4; q += blockDim.x) {
            const int p = 4 * q, r = p / a.W, c = p - r * a.W;
            const int* m = smap + r * pitch + c;
            o4[q] = make_int4(finish(a, m[0]), finish(a, m[1]), finish(a, m[2]), finish(a, m[3]));
        }
    } else {
        for (int p = threadIdx.x; p < a.N; p += blockDim.x) {
            const int r = p / a.W, c = p - r * a.W;
            out[p] = finish(a, smap[r * pitch + c]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.convert && src >= 0 && KIND == 1 && !a.f[src]) out[src] = 0;
}

// Map in global memory (the output row itself), for images whose map does
// not fit in shared memory.
template <int CONN, int KIND, int VPL>
__global__ void __launch_bounds__(32 * PWARPS) k_propagate_glob(PropArgs a) {
    __shared__ int s_flag[2], s_rounds;
    const int j = blockIdx.x;
    const int njobs = a.njobs_dev ? *a.njobs_dev : a.njobs;
    if (j >= njobs) return;
    const int src = a.sources ? a.sources[j] : -1;
    int* map = a.map_base + (size_t)(a.map_row ? a.map_row[j] : j) * (size_t)a.N;
    for (int p = threadIdx.x; p < a.N; p += blockDim.x) map[p] = is_seed(a, src, p) ? 0 : PINF;
    if (threadIdx.x == 0) { s_flag[0] = 0; s_flag[1] = 0; }
    __threadfence_block();
    __syncthreads();
    const GlobMap gm{map, a.W};
    run_block<CONN, KIND, VPL>(a, gm, s_flag, &s_rounds);
    __syncthreads();
    if (threadIdx.x == 0 && a.sweeps) atomicAdd(a.sweeps, (unsigned long long)s_rounds * PWARPS);
    if (a.convert) {
        for (int p = threadIdx.x; p < a.N; p += blockDim.x) {
            const int v = ld_cg(map + p);
            if (v >= PINF) map[p] = (int)UNREACH;
        }
        __syncthreads();
        if (threadIdx.x == 0 && src >= 0 && KIND == 1 && !a.f[src]) map[src] = 0;
    }
}

constexpr int SMEM_MAP_LIMIT = 200 * 1024;

template <int CONN, int KIND, int VPL>
cudaError_t launch_one(const PropArgs& a, int jobs, cudaStream_t st) {
    const int pitch = a.W | 1;  // odd pitch: row and column lines avoid bank conflicts
    const size_t smem = (size_t)a.H * pitch * sizeof(int);
    if (smem <= (size_t)SMEM_MAP_LIMIT) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_propagate_smem<CONN, KIND, VPL>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_MAP_LIMIT);
            attr = true;
        }
        k_propagate_smem<CONN, KIND, VPL><<<jobs, 32 * PWARPS, smem, st>>>(a, pitch);
    } else {
        k_propagate_glob<CONN, KIND, VPL><<<jobs, 32 * PWARPS, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int CONN, int KIND>
cudaError_t launch_vpl(const PropArgs& a, int vpl, int jobs, cudaStream_t st) {
    switch (vpl) {
        case 1: return launch_one<CONN, KIND, 1>(a, jobs, st);
        case 2: return launch_one<CONN, KIND, 2>(a, jobs, st);
        case 4: return launch_one<CONN, KIND, 4>(a, jobs, st);
        case 8: return launch_one<CONN, KIND, 8>(a, jobs, st);
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
    const int vpl = prop_vpl(a.H > a.W ? a.H : a.W);
    const int jobs = grid * wpb;  // one block per job
    if (jobs <= 0) return cudaSuccess;
    if (conn == 8) return kind == 0 ? launch_vpl<8, 0>(a, vpl, jobs, st) : launch_vpl<8, 1>(a, vpl, jobs, st);
    return kind == 0 ? launch_vpl<4, 0>(a, vpl, jobs, st) : launch_vpl<4, 1>(a, vpl, jobs, st);
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
