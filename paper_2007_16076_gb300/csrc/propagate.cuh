// Kernel (a): geodesic propagation on the image graph (templates; each
// propagate_k<KIND>.cu instantiates one edge-cost kind).
//
// Computes d(s, .) = min over paths of the summed edge weights (Sec. 2, eqs.
// "temps" and "distance"), the "geodesic time function" of Soille that the
// paper uses with a 3x3 neighbourhood (Sec. 3). Weights are w(p,q) = f(p) +
// f(q) + 1 (grey: the sum of grey levels), |f(p) - f(q)| + 1 (the L1
// pseudo-metric) or 2 between free pixels (mask). KIND 0 / 2 / 1.
//
// One block owns one source (or one multi-source seed set). Its distance
// map sits in shared memory (global memory for images too large), set to 0
// at the seeds and "unreached" elsewhere, next to two copies of the image
// (row-major and column-major). Warps sweep the map concurrently, each in
// its own direction (rows top-down, rows bottom-up, columns left-right,
// columns right-left); when a direction has two or four warps, each sweeps
// an equal contiguous share of its lines every round, starting from the
// line before its share as it stands. For each line a warp
//   1. relaxes every pixel from the previous line it just finished (the
//      three neighbours behind it for 8-connectivity, one for 4), then
//   2. closes the line inside each lane: lane j holds pixels VPL*j ..
//      VPL*j+VPL-1 and, with P the prefix sum of the line's edge weights,
//      takes min_c' v(c') + |P(c) - P(c')| over its own pixels (a prefix-min
//      of v - P and a suffix-min of v + P). Values cross lane boundaries
//      through the sweeps of the other axis; a full warp-wide scan on every
//      line measured slower,
// and lowers the map with atomic minima, flagging every line that a lowered
// pixel belongs to (its own line and the crossing one). After the first
// rounds most lines stop changing, and a warp skips a line when neither it
// nor the line before it was flagged in the previous round.
//
// Every stored value is the cost of a real path, so values only decrease
// towards the distances; weights are positive integers, so the fixpoint is
// unique and any schedule reaches it. The block stops after a round (one
// pass per warp) in which no warp lowered anything: the map was constant
// while every edge direction was tested. Rounds are capped; hitting the cap
// sets a status bit instead of looping on.
#pragma once
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace gapsp {

namespace {

constexpr int MAXWARPS = 16;              // 4 directions x up to 4 phases

// KIND 0 (grey) and 3 (sum of the channels of a multichannel image) weigh
// an edge by the sum of its ends' levels; KIND 3's levels are 16-bit.
__host__ __device__ constexpr bool sum_kind(int k) { return k == 0 || k == 3; }
template <int KIND>
using Level = typename std::conditional<KIND == 3, uint16_t, uint8_t>::type;
template <int KIND>
__device__ __forceinline__ int level_at(const uint8_t* f, int p) {
    return KIND == 3 ? (int)__ldg(reinterpret_cast<const uint16_t*>(f) + p) : (int)__ldg(f + p);
}
constexpr int BIGX = PINF;                // identity of the prefix-min of v - P
constexpr int BIGY = PINF + (1 << 18);    // identity of the suffix-min of v + P

// Where element x of a line sits in shared memory. Lane j holds elements
// VPL*j .. VPL*j + VPL - 1 of a line, so element k of the 32 lanes would be
// VPL words apart and fall into 32 / VPL banks only; rotating each lane's
// group of VPL elements by x / 32 spreads them over all 32 banks. The map
// stores pixel (r, c) at swz(r) * pitch + swz(c) (odd pitch): element k of
// a row line (consecutive words) and of a column line (rows pitch apart)
// then sits in a different bank for every lane. Lines are padded to a
// multiple of VPL so that the rotation stays inside the storage.
template <int VPL>
__host__ __device__ __forceinline__ int swz(int x) {
    return VPL == 1 ? x : ((x & ~(VPL - 1)) | ((x + (x >> 5)) & (VPL - 1)));
}

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <int VPL>
struct SmemMap {
    int* base;
    int pitch;
    __device__ __forceinline__ int* at(int r, int c) const { return base + swz<VPL>(r) * pitch + swz<VPL>(c); }
    __device__ __forceinline__ int ld(int r, int c) const { return *((volatile const int*)at(r, c)); }
    __device__ __forceinline__ void lower(int r, int c, int v) const { atomicMin(at(r, c), v); }
};

struct GlobMap {
    int* base;
    int pitch;
    __device__ __forceinline__ int ld(int r, int c) const { return ld_cg(base + r * pitch + c); }
    __device__ __forceinline__ void lower(int r, int c, int v) const { atomicMin(base + r * pitch + c, v); }
};

// Shared state of one block besides the map. A block owns the strip of rows
// [r0, r0 + hs) of the image (the whole image unless the source is split
// over a cluster of blocks).
struct Shared {
    const void* fR;     // strip of the image's levels, row-major [hs][W]
    const void* fC;     // strip of the image's levels, column-major [W][hs]
    uint8_t* chR;       // [3][hs]: row line lowered during round t (slot t % 3)
    uint8_t* chC;       // [3][W]: column line lowered during round t
    int r0, hs;
    int pitch;                // map pitch of every strip of the cluster (shared memory)
    // rows next to the strip, owned by the neighbour blocks of the cluster
    // (distributed shared memory), or NULL at the image border
    const int* up_map;        // neighbour above: its map; its last row is row r0 - 1
    const uint8_t* up_chR;    // its row flags
    int up_hs;
    const int* dn_map;        // neighbour below: its map; its first row is row r0 + hs
    const uint8_t* dn_chR;
    int dn_hs;
};

// One pass over all lines in one direction during round `round`; true if
// this warp lowered some value. A line is skipped when neither it nor the
// line before it was lowered during the previous round: by induction over
// rounds, the last result of this warp on it still satisfies every edge
// this direction tests (the flags of a round are read only after the
// block barrier that ends it).
// VPL grey levels of one lane, from a VPL-aligned address in shared memory.
template <int VPL, class Lv>
__device__ __forceinline__ void load_levels(const Lv* p, int (&fc)[VPL]) {
    if constexpr (sizeof(Lv) != 1) {
#pragma unroll
        for (int k = 0; k < VPL; ++k) fc[k] = p[k];
    } else if constexpr (VPL == 4) {
        const uchar4 u = *reinterpret_cast<const uchar4*>(p);
        fc[0] = u.x; fc[1] = u.y; fc[2] = u.z; fc[3] = u.w;
    } else if constexpr (VPL == 2) {
        const uchar2 u = *reinterpret_cast<const uchar2*>(p);
        fc[0] = u.x; fc[1] = u.y;
    } else {
#pragma unroll
        for (int k = 0; k < VPL; ++k) fc[k] = p[k];
    }
}

// EX: every line is exactly 32 * VPL pixels long (square single-block
// images such as 128 x 128 with VPL = 4), so no lane holds a pixel past the
// end of a line and the bounds tests drop out.
template <int CONN, int KIND, int VPL, bool ROWS, bool EX, class Map>
__device__ bool sweep(const PropArgs& a, const Map& map, const Shared& sh, int dir, int start, int lane,
                      int round, int& nproc, int seg) {
    const int nlines = ROWS ? sh.hs : a.W;
    const int len = ROWS ? a.W : sh.hs;
    using Lv = Level<KIND>;
    const Lv* f_line = static_cast<const Lv*>(ROWS ? sh.fR : sh.fC);
    uint8_t* ch_own = (ROWS ? sh.chR : sh.chC) + (round % 3) * nlines;
    uint8_t* ch_x = (ROWS ? sh.chC : sh.chR) + (round % 3) * len;
    const uint8_t* prev_own = (ROWS ? sh.chR : sh.chC) + ((round + 2) % 3) * nlines;
    const int wrap_at = dir > 0 ? 0 : nlines - 1;  // a sweep restarts here
    // gp[k]: cost of leaving the previous line's pixel, d + f (grey) or d
    // (mask, L1); gf[k]: its grey level (L1)
    int gp[VPL], gf[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        gp[k] = PINF;
        gf[k] = 0;
    }
    bool has_pred = false;      // this line has a previous line in the sweep
    bool pred_changed = false;  // the previous line changed (it must be relaxed from)
    bool changed = false;
    int l = start;
    for (int i = 0; i < seg; ++i) {
        if (i == 0 || l == wrap_at) {
            // (re)start: the previous line is the neighbour block's edge row
            // when the sweep enters the strip from a split border, else none
            has_pred = false;
            pred_changed = false;
#pragma unroll
            for (int k = 0; k < VPL; ++k) gp[k] = PINF;
            if (ROWS) {
                const int* rmap = nullptr;
                const uint8_t* rch = nullptr;
                int rrow = 0, rhs = 1, grow = 0;
                if (dir > 0 && l == 0 && sh.up_map) {
                    rmap = sh.up_map; rch = sh.up_chR; rhs = sh.up_hs; rrow = rhs - 1; grow = sh.r0 - 1;
                } else if (dir < 0 && l == nlines - 1 && sh.dn_map) {
                    rmap = sh.dn_map; rch = sh.dn_chR; rhs = sh.dn_hs; rrow = 0; grow = sh.r0 + sh.hs;
                }
                if (rmap) {
                    has_pred = true;
                    pred_changed = rch[((round + 2) % 3) * rhs + rrow] != 0 ||
                                   *((volatile const uint8_t*)(rch + (round % 3) * rhs + rrow)) != 0;
#pragma unroll
                    for (int k = 0; k < VPL; ++k) {
                        const int pos = VPL * lane + k;
                        const int dv =
                            pos < len ? *((volatile const int*)(rmap + swz<VPL>(rrow) * sh.pitch + swz<VPL>(pos)))
                                      : PINF;
                        const int fg = pos < len ? level_at<KIND>(a.f, grow * a.W + pos) : 0;
                        gp[k] = sum_kind(KIND) ? (pos < len ? dv + fg : dv) : KIND == 2 ? dv : (fg ? dv : PINF);
                        gf[k] = fg;
                    }
                }
            }
        }
        if (i == 0 && l != wrap_at) {
            // the warp's share of the lines starts inside the image: relax
            // from the line before it, as it stands now
            const int lp = l - dir;
            has_pred = true;
            pred_changed = prev_own[lp] != 0 || *((volatile const uint8_t*)(ch_own + lp)) != 0;
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                const int pos = VPL * lane + k;
                const int dv = (EX || pos < len) ? (ROWS ? map.ld(lp, pos) : map.ld(pos, lp)) : PINF;
                const int fp = (EX || pos < len) ? (int)f_line[lp * len + pos] : 0;
                gp[k] = sum_kind(KIND) ? dv + fp : KIND == 2 ? dv : (fp ? dv : PINF);
                gf[k] = fp;
            }
        }
        // lowered in the previous round, or already in this one (seen so far);
        // before the first round the lines holding a seed count as lowered
        const bool own_changed = prev_own[l] != 0 || *((volatile const uint8_t*)(ch_own + l)) != 0;
        const bool skip = !own_changed && !(has_pred && pred_changed);
        int fc[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int pos = VPL * lane + k;
            if (!EX) fc[k] = pos < len ? f_line[l * len + pos] : 0;
        }
        if (EX) load_levels<VPL>(f_line + l * len + VPL * lane, fc);
        if (skip) {
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                const int pos = VPL * lane + k;
                const int dv = (EX || pos < len) ? (ROWS ? map.ld(l, pos) : map.ld(pos, l)) : PINF;
                gp[k] = sum_kind(KIND) ? dv + fc[k] : KIND == 2 ? dv : (fc[k] ? dv : PINF);
                gf[k] = fc[k];
            }
            has_pred = true;
            pred_changed = false;
            l += dir;
            if (l < 0) l += nlines;
            if (l >= nlines) l -= nlines;
            continue;
        }
        int o[VPL], p[VPL];
        bool freep[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int pos = VPL * lane + k;
            const bool valid = EX || pos < len;
            o[k] = valid ? (ROWS ? map.ld(l, pos) : map.ld(pos, l)) : PINF;
            freep[k] = valid && (KIND != 1 || fc[k] != 0);
        }
        if (KIND != 1) {
            // prefix of the line's edge weights from the lane's first pixel
            // (only differences inside a lane are used)
            int acc = 0;
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                p[k] = acc;
                if (k + 1 < VPL) acc += (sum_kind(KIND) ? fc[k] + fc[k + 1] : abs(fc[k + 1] - fc[k])) + 1;
            }
        } else {
#pragma unroll
            for (int k = 0; k < VPL; ++k) p[k] = 2 * k;
        }
        // 1. relax from the previous line
        int gl0 = PINF, gr0 = PINF, fl0 = 0, fr0 = 0;
        if (CONN == 8) {
            gl0 = __shfl_up_sync(FULL, gp[VPL - 1], 1);
            gr0 = __shfl_down_sync(FULL, gp[0], 1);
            if (KIND == 2) {
                fl0 = __shfl_up_sync(FULL, gf[VPL - 1], 1);
                fr0 = __shfl_down_sync(FULL, gf[0], 1);
            }
            if (lane == 0) gl0 = PINF;
            if (lane == 31) gr0 = PINF;
        }
        int v[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            int best;
            if (KIND == 2) {
                // L1: the weight depends on both ends of the edge
                int g = gp[k] + abs(gf[k] - fc[k]) + 1;
                if (CONN == 8) {
                    const int gl = k > 0 ? gp[k - 1] : gl0, fl = k > 0 ? gf[k - 1] : fl0;
                    const int gr = k + 1 < VPL ? gp[k + 1] : gr0, fr = k + 1 < VPL ? gf[k + 1] : fr0;
                    g = min(g, min(gl + abs(fl - fc[k]) + 1, gr + abs(fr - fc[k]) + 1));
                }
                best = min(o[k], g);
            } else {
                int g = gp[k];
                if (CONN == 8) {
                    const int gl = k > 0 ? gp[k - 1] : gl0;
                    const int gr = k + 1 < VPL ? gp[k + 1] : gr0;
                    g = min(g, min(gl, gr));
                }
                best = min(o[k], g + (sum_kind(KIND) ? fc[k] + 1 : 2));
            }
            v[k] = freep[k] ? best : PINF;
        }
        // 2. close the line inside each lane
        int sx[VPL], sy[VPL], d[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int x = freep[k] ? v[k] - p[k] : BIGX;
            sx[k] = (KIND == 1 && !freep[k]) ? BIGX : min(k > 0 ? sx[k - 1] : BIGX, x);
        }
#pragma unroll
        for (int k = VPL - 1; k >= 0; --k) {
            const int y = freep[k] ? v[k] + p[k] : BIGY;
            sy[k] = (KIND == 1 && !freep[k]) ? BIGY : min(k + 1 < VPL ? sy[k + 1] : BIGY, y);
        }
#pragma unroll
        for (int k = 0; k < VPL; ++k)
            d[k] = freep[k] ? min(v[k], min(sx[k] + p[k], sy[k] - p[k])) : PINF;
        // lower the map where this line improved, then bump the versions of
        // this line and of every crossing line that changed
        bool mine = false;
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            if (freep[k] && d[k] < o[k]) {
                mine = true;
                const int pos = VPL * lane + k;
                if (ROWS) map.lower(l, pos, d[k]);
                else map.lower(pos, l, d[k]);
            }
            gp[k] = sum_kind(KIND) ? d[k] + fc[k] : d[k];
            gf[k] = fc[k];
        }
        ++nproc;
        if (mine) {
#pragma unroll
            for (int k = 0; k < VPL; ++k)
                if (freep[k] && d[k] < o[k]) ch_x[VPL * lane + k] = 1;
            ch_own[l] = 1;
            changed = true;
        }
        has_pred = true;
        pred_changed = own_changed || __any_sync(FULL, mine);
        l += dir;
        if (l < 0) l += nlines;
        if (l >= nlines) l -= nlines;
    }
    return changed;
}

template <int CONN, int KIND, int VPL, class Map, bool CL, bool EX>
__device__ void run_block(const PropArgs& a, const Map& map, const Shared& sh, int* s_flag, int* s_rounds) {
    const int nr = sh.hs, nc = a.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dirk = warp & 3, phase = warp >> 2, nph = blockDim.x >> 7;
    const bool rows = dirk < 2;
    const int dir = (dirk & 1) ? -1 : +1;
    const int nlines = rows ? sh.hs : a.W;
    // the warps of one direction share its lines: each sweeps an equal,
    // contiguous part of them every round
    const int off = (phase * nlines) / nph;
    const int start = dir > 0 ? off : (nlines - 1 - off);
    const int seg = ((phase + 1) * nlines) / nph - off;
    int round = 0, nproc = 0;
    for (;;) {
        // clear the flag slot the next round will write (last used two rounds ago)
        const int nx = (round + 1) % 3;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) sh.chR[nx * nr + i] = 0;
        for (int i = threadIdx.x; i < nc; i += blockDim.x) sh.chC[nx * nc + i] = 0;
        bool ch;
        if (rows) ch = sweep<CONN, KIND, VPL, true, EX, Map>(a, map, sh, dir, start, lane, round, nproc, seg);
        else ch = sweep<CONN, KIND, VPL, false, EX, Map>(a, map, sh, dir, start, lane, round, nproc, seg);
        ch = __any_sync(FULL, ch);
        if (lane == 0 && ch) s_flag[round & 1] = 1;
        bool any;
        if (CL) {
            // every block of the cluster has finished the round
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            any = false;
            for (unsigned r = 0; r < cl.num_blocks(); ++r)
                any |= *((volatile int*)cl.map_shared_rank(s_flag + (round & 1), r)) != 0;
        } else {
            __syncthreads();
            any = s_flag[round & 1] != 0;
        }
        if (threadIdx.x == 0) s_flag[(round + 1) & 1] = 0;
        ++round;
        if (!any) break;
        if (round * 4 >= a.max_sweeps) {
            if (threadIdx.x == 0) atomicOr(a.status, ST_NOT_CONVERGED);
            break;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *s_rounds = round;
    if (lane == 0 && a.sweeps) atomicAdd(a.sweeps + (S_LINES - S_SWEEPS), (unsigned long long)nproc);
}

__device__ __forceinline__ int finish(const PropArgs& a, int v) {
    return (a.convert && v >= PINF) ? (int)UNREACH : v;
}

// Seeds start at 0. On a mask, an obstacle pixel is never a seed: a source
// on an obstacle reaches nothing (its own entry is set to 0 at the end).
__device__ __forceinline__ bool is_seed(const PropArgs& a, int src, int p) {
    const bool s = a.seed_flags ? a.seed_flags[p] != 0 : p == src;
    return s && (!a.kind_mask || a.f[p] != 0);
}

// Flags of the strip's lines, then its levels row- and column-major.
__host__ __device__ inline size_t shared_state_bytes(int hs, int W, int level_bytes) {
    return ((3 * (size_t)(hs + W) + 2 * (size_t)hs * W * level_bytes) + 15) & ~(size_t)15;
}

// Lays out the non-map shared state of the strip [r0, r0 + hs) after `base`
// and initialises it.
template <int KIND, int VPL>
__device__ Shared setup_shared(const PropArgs& a, char* base, int r0, int hs) {
    Shared sh{};
    sh.r0 = r0;
    sh.hs = hs;
    uint8_t* bp = reinterpret_cast<uint8_t*>(base);
    sh.chR = bp;
    sh.chC = bp + 3 * hs;
    using Lv = Level<KIND>;
    // the levels start on an even offset (16-bit levels)
    Lv* fR = reinterpret_cast<Lv*>(bp + ((3 * (hs + a.W) + 1) & ~1));
    Lv* fC = fR + hs * a.W;
    for (int p = threadIdx.x; p < hs * a.W; p += blockDim.x) {
        const int r = p / a.W, c = p - r * a.W;
        const Lv v = (Lv)level_at<KIND>(a.f, (r0 + r) * a.W + c);
        fR[p] = v;
        fC[c * hs + r] = v;
    }
    for (int i = threadIdx.x; i < 3 * (hs + a.W); i += blockDim.x) bp[i] = 0;
    sh.fR = fR;
    sh.fC = fC;
    return sh;
}

// Before the first round, the lines that hold a seed are the only ones
// whose values differ from "unreached" (flag slot 2 is the one round 0
// reads as "previous round").
__device__ void flag_seed_lines(const PropArgs& a, const Shared& sh, int src) {
    if (a.seed_flags) {
        for (int p = threadIdx.x; p < sh.hs * a.W; p += blockDim.x)
            if (a.seed_flags[sh.r0 * a.W + p]) {
                const int r = p / a.W, c = p - r * a.W;
                sh.chR[2 * sh.hs + r] = 1;
                sh.chC[2 * a.W + c] = 1;
            }
    } else if (threadIdx.x == 0 && src >= 0) {
        const int r = src / a.W - sh.r0, c = src % a.W;
        if (r >= 0 && r < sh.hs) {
            sh.chR[2 * sh.hs + r] = 1;
            sh.chC[2 * a.W + c] = 1;
        }
    }
}

// Warm start. During a fill every entry of D is UNREACH (set before the
// first round) or the cost of a real path, exact once the pair is filled:
// the fills and the propagations write nothing else. Any entry therefore
// bounds its distance from above, even one read while another launch is
// writing it (the old and the new value are both bounds), and so do the
// sums d(s,q) + d(q,x) over a neighbour q of s (triangle inequality). The
// map of source s starts from the least of these bounds instead of
// "unreached": the sweeps reach the same unique fixpoint from any upper
// bounds, and most pairs of a late source are filled already. Warp 0 picks
// the neighbours whose d(s,q) is known (axial first); returns how many.
constexpr int MAXHELP = 8;
struct Helpers {
    const uint32_t* row[MAXHELP];  // row q of D
    int d[MAXHELP];                // bound of d(s, q)
    int n;
};

__device__ int pick_helpers(const PropArgs& a, int src, Helpers& h) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        bool ok = false;
        const uint32_t* row = nullptr;
        int dq = 0;
        if (a.warm_rows && src >= 0 && lane < a.conn && (!a.kind_mask || a.f[src])) {
            const int r = src / a.W, c = src - r * a.W;
            const int rr = r + (lane < 4 ? (lane == 0 ? -1 : lane == 1 ? 1 : 0) : (lane < 6 ? -1 : 1));
            const int cc = c + (lane < 4 ? (lane == 2 ? -1 : lane == 3 ? 1 : 0) : ((lane & 1) ? 1 : -1));
            if (rr >= 0 && rr < a.H && cc >= 0 && cc < a.W) {
                const int q = rr * a.W + cc;
                const uint32_t v = __ldcg(a.warm_rows + (size_t)src * a.N + q);
                if (v < (uint32_t)PINF && (!a.kind_mask || a.f[q])) {
                    ok = true;
                    row = a.warm_rows + (size_t)q * a.N;
                    dq = (int)v;
                }
            }
        }
        const unsigned m = __ballot_sync(FULL, ok);
        if (ok) {
            const int i = __popc(m & ((1u << lane) - 1u));
            h.row[i] = row;
            h.d[i] = dq;
        }
        if (lane == 0) h.n = __popc(m);
    }
    __syncthreads();
    return h.n;
}

__device__ __forceinline__ int warm_bound(uint32_t dx, int dq) {
    // both terms are below PINF (< 2^30), so the sum fits; a bound above
    // PINF is no bound
    return dx < (uint32_t)PINF ? min((int)dx + dq, PINF) : PINF;
}

// The strip's map before the first round: the seeds at 0, elsewhere
// "unreached" or, warm, the least bound from row s and the neighbours' rows
// (obstacles stay unreached). Warm, a line is flagged for the first round
// when it holds a finite value (flag slot 2 is the one round 0 reads as
// "previous round"); returns whether the map is warm.
template <int KIND, int VPL>
__device__ bool init_map(const PropArgs& a, int* smap, int pitch, uint8_t* flags, int r0, int hs, int src,
                         const Helpers& h, int nh) {
    const SmemMap<VPL> map{smap, pitch};
    const int n = hs * a.W, g0 = r0 * a.W;
    const bool warm = a.warm_rows && src >= 0;
    if (!warm) {
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int r = p / a.W, c = p - r * a.W;
            *map.at(r, c) = is_seed(a, src, g0 + p) ? 0 : PINF;
        }
        return false;
    }
    uint8_t* fr = flags + 2 * hs;            // row lines of the strip
    uint8_t* fc = flags + 3 * hs + 2 * a.W;  // column lines
    const uint32_t* own = a.warm_rows + (size_t)src * a.N + g0;
    if ((a.W & 3) == 0) {
        // rows start on 16-byte boundaries (the array is 16-byte aligned)
        for (int p = 4 * threadIdx.x; p < n; p += 4 * blockDim.x) {
            const uint4 u0 = __ldcg(reinterpret_cast<const uint4*>(own + p));
            int v[4] = {warm_bound(u0.x, 0), warm_bound(u0.y, 0), warm_bound(u0.z, 0), warm_bound(u0.w, 0)};
            for (int k = 0; k < nh; ++k) {
                const uint4 u = __ldcg(reinterpret_cast<const uint4*>(h.row[k] + g0 + p));
                v[0] = min(v[0], warm_bound(u.x, h.d[k]));
                v[1] = min(v[1], warm_bound(u.y, h.d[k]));
                v[2] = min(v[2], warm_bound(u.z, h.d[k]));
                v[3] = min(v[3], warm_bound(u.w, h.d[k]));
            }
            const int r = p / a.W, c = p - r * a.W;  // 4 pixels of one row (W % 4 = 0)
            bool any = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int x = v[k];
                if (KIND == 1 && !a.f[g0 + p + k]) x = PINF;
                if (is_seed(a, src, g0 + p + k)) x = 0;
                *map.at(r, c + k) = x;
                if (x < PINF) {
                    any = true;
                    fc[c + k] = 1;
                }
            }
            if (any) fr[r] = 1;
        }
    } else {
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            int x = warm_bound(__ldcg(own + p), 0);
            for (int k = 0; k < nh; ++k) x = min(x, warm_bound(__ldcg(h.row[k] + g0 + p), h.d[k]));
            if (KIND == 1 && !a.f[g0 + p]) x = PINF;
            if (is_seed(a, src, g0 + p)) x = 0;
            const int r = p / a.W, c = p - r * a.W;
            *map.at(r, c) = x;
            if (x < PINF) {
                fr[r] = 1;
                fc[c] = 1;
            }
        }
    }
    return true;
}

// Map in shared memory. One block per job, or a cluster of C blocks per job
// (CL), each owning a strip of rows; the strips see each other's edge rows
// through distributed shared memory.
template <int CONN, int KIND, int VPL, bool CL, bool EX>
__global__ void __launch_bounds__(32 * MAXWARPS) k_propagate_smem(PropArgs a, int pitch, int C) {
    extern __shared__ int smap[];
    pdl_trigger();  // the tree launch that follows may be scheduled
    __shared__ int s_flag[2], s_rounds;
    const int j = blockIdx.x / C, rank = blockIdx.x % C;
    const int njobs = a.njobs_dev ? *a.njobs_dev : a.njobs;
    if (j >= njobs) return;  // the whole cluster leaves together
    const int hs0 = (a.H + C - 1) / C;
    const int r0 = rank * hs0, hs = min(hs0, a.H - r0);
    const int src = a.sources ? a.sources[j] : -1;
    // a row computed ahead of its round is not computed again (no launch that
    // may run concurrently with this one writes this source's flag, so the
    // blocks of a cluster all see the same value and leave together)
    if (a.row_done && src >= 0 && a.row_done[src]) {
        if (a.hits && threadIdx.x == 0 && rank == 0) atomicAdd(a.hits, 1ull);
        return;
    }
    int* out = a.map_base + (size_t)(a.map_row ? a.map_row[j] : j) * (size_t)a.N;
    __shared__ Helpers s_help;
    const int nh = pick_helpers(a, src, s_help);
    // the flags are cleared by setup_shared: it comes first, then the map
    // every strip's map has the same padded height, so the state after it
    // sits at the same offset in every block of the cluster
    const int rows = round_up(hs0, VPL);
    Shared sh = setup_shared<KIND, VPL>(a, reinterpret_cast<char*>(smap + rows * pitch), r0, hs);
    sh.pitch = pitch;
    if (threadIdx.x == 0) { s_flag[0] = 0; s_flag[1] = 0; }
    __syncthreads();
    const bool warm = init_map<KIND, VPL>(a, smap, pitch, sh.chR, r0, hs, src, s_help, nh);
    if (!warm) flag_seed_lines(a, sh, src);
    if (CL) {
        cg::cluster_group cl = cg::this_cluster();
        if (rank > 0) {
            sh.up_map = cl.map_shared_rank(smap, rank - 1);
            sh.up_hs = hs0;
            sh.up_chR = reinterpret_cast<const uint8_t*>(sh.up_map + rows * pitch);
        }
        if (rank + 1 < C) {
            sh.dn_map = cl.map_shared_rank(smap, rank + 1);
            sh.dn_hs = min(hs0, a.H - (rank + 1) * hs0);
            sh.dn_chR = reinterpret_cast<const uint8_t*>(sh.dn_map + rows * pitch);
        }
        cl.sync();  // every strip is initialised before any remote access
    } else {
        __syncthreads();
    }
    const SmemMap<VPL> map{smap, pitch};
    run_block<CONN, KIND, VPL, SmemMap<VPL>, CL, EX>(a, map, sh, s_flag, &s_rounds);
    if (CL) cg::this_cluster().sync();  // no block leaves while others may read it
    __syncthreads();
    if (threadIdx.x == 0 && a.sweeps) atomicAdd(a.sweeps, (unsigned long long)s_rounds * (blockDim.x >> 5));
    // finished strip of the row: coalesced 128-bit stores
    const int n = hs * a.W;
    int* o = out + (size_t)r0 * a.W;
    if ((a.W & 3) == 0) {
        int4* o4 = reinterpret_cast<int4*>(o);
        for (int q = threadIdx.x; q < n / 4; q += blockDim.x) {
            const int p = 4 * q, r = p / a.W, c = p - r * a.W;
            o4[q] = make_int4(finish(a, *map.at(r, c)), finish(a, *map.at(r, c + 1)), finish(a, *map.at(r, c + 2)),
                              finish(a, *map.at(r, c + 3)));
        }
    } else {
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int r = p / a.W, c = p - r * a.W;
            o[p] = finish(a, *map.at(r, c));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.convert && src >= 0 && KIND == 1 && !a.f[src] && src / a.W >= r0 &&
        src / a.W < r0 + hs)
        out[src] = 0;
    if (threadIdx.x == 0 && rank == 0 && a.row_done && src >= 0) {
        a.row_done[src] = 1;  // read by later launches only
        if (a.ran) atomicAdd(a.ran, 1ull);
    }
}

// Map in global memory (the output row itself), for images whose map does
// not fit in shared memory.
template <int CONN, int KIND, int VPL>
__global__ void __launch_bounds__(32 * MAXWARPS) k_propagate_glob(PropArgs a) {
    extern __shared__ int sbuf[];
    pdl_trigger();
    __shared__ int s_flag[2], s_rounds;
    const int j = blockIdx.x;
    const int njobs = a.njobs_dev ? *a.njobs_dev : a.njobs;
    if (j >= njobs) return;
    const int src = a.sources ? a.sources[j] : -1;
    if (a.row_done && src >= 0 && a.row_done[src]) {
        if (a.hits && threadIdx.x == 0) atomicAdd(a.hits, 1ull);
        return;
    }
    int* map = a.map_base + (size_t)(a.map_row ? a.map_row[j] : j) * (size_t)a.N;
    for (int p = threadIdx.x; p < a.N; p += blockDim.x) map[p] = is_seed(a, src, p) ? 0 : PINF;
    const Shared sh = setup_shared<KIND, VPL>(a, reinterpret_cast<char*>(sbuf), 0, a.H);
    if (threadIdx.x == 0) { s_flag[0] = 0; s_flag[1] = 0; }
    __threadfence_block();
    __syncthreads();
    flag_seed_lines(a, sh, src);
    __syncthreads();
    const GlobMap gm{map, a.W};
    run_block<CONN, KIND, VPL, GlobMap, false, false>(a, gm, sh, s_flag, &s_rounds);
    __syncthreads();
    if (threadIdx.x == 0 && a.sweeps) atomicAdd(a.sweeps, (unsigned long long)s_rounds * (blockDim.x >> 5));
    if (a.convert) {
        for (int p = threadIdx.x; p < a.N; p += blockDim.x) {
            const int v = ld_cg(map + p);
            if (v >= PINF) map[p] = (int)UNREACH;
        }
        __syncthreads();
        if (threadIdx.x == 0 && src >= 0 && KIND == 1 && !a.f[src]) map[src] = 0;
    }
    if (threadIdx.x == 0 && a.row_done && src >= 0) {
        a.row_done[src] = 1;  // read by later launches only
        if (a.ran) atomicAdd(a.ran, 1ull);
    }
}

constexpr int SMEM_LIMIT = 220 * 1024;

// Map pitch: the width padded to a multiple of the values per lane, odd.
int map_pitch(const PropArgs& a) { return round_up(a.W, prop_vpl(a.H > a.W ? a.H : a.W)) | 1; }

size_t smem_for_strips(const PropArgs& a, int c) {
    const int hs = (a.H + c - 1) / c;
    const int rows = round_up(hs, prop_vpl(a.H > a.W ? a.H : a.W));
    return (size_t)rows * map_pitch(a) * sizeof(int) + shared_state_bytes(hs, a.W, a.level_bytes) + 16;
}

// Row strips (blocks of one cluster) per source: the requested cluster size,
// halved while a strip would be shorter than 8 rows, doubled while a strip
// does not fit in shared memory; 0 when even 8 strips do not fit (the map
// then lives in global memory, one block per source).
int strips_per_job(const PropArgs& a) {
    int C = a.cluster > 0 ? a.cluster : 1;
    while (C > 1 && a.H / C < 8) C >>= 1;
    while (smem_for_strips(a, C) > (size_t)SMEM_LIMIT && C < 8 && a.H / (2 * C) >= 1) C <<= 1;
    return smem_for_strips(a, C) <= (size_t)SMEM_LIMIT ? C : 0;
}

template <int CONN, int KIND, int VPL>
cudaError_t launch_one(const PropArgs& a, int jobs, cudaStream_t st) {
    const int pitch = map_pitch(a);
    const int threads = 32 * 4 * (a.phases == 4 ? 4 : a.phases == 2 ? 2 : 1);
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_propagate_smem<CONN, KIND, VPL, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
        cudaFuncSetAttribute(k_propagate_smem<CONN, KIND, VPL, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
        cudaFuncSetAttribute(k_propagate_smem<CONN, KIND, VPL, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
        cudaFuncSetAttribute(k_propagate_glob<CONN, KIND, VPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_LIMIT);
    });
    const int C = strips_per_job(a);
    if (C > 0) {
        const size_t smem = smem_for_strips(a, C);
        if (C == 1) {
            if (a.W == 32 * VPL && a.H == 32 * VPL)
                k_propagate_smem<CONN, KIND, VPL, false, true><<<jobs, threads, smem, st>>>(a, pitch, 1);
            else
                k_propagate_smem<CONN, KIND, VPL, false, false><<<jobs, threads, smem, st>>>(a, pitch, 1);
        } else {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(jobs * C);
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, k_propagate_smem<CONN, KIND, VPL, true, false>, a, pitch, C);
            if (e != cudaSuccess) return e;
        }
    } else {
        const size_t state = shared_state_bytes(a.H, a.W, a.level_bytes) + 16;
        if (state > (size_t)SMEM_LIMIT) return cudaErrorInvalidValue;
        k_propagate_glob<CONN, KIND, VPL><<<jobs, threads, state, st>>>(a);
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

// The launches of one edge-cost kind, 4- or 8-connected (propagate_k<KIND>.cu).
cudaError_t launch_k0(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st);
cudaError_t launch_k1(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st);
cudaError_t launch_k2(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st);
cudaError_t launch_k3(const PropArgs& a, int conn, int vpl, int jobs, cudaStream_t st);

}  // namespace gapsp
