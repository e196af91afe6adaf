// Kernel (c): choice of the next sources, and the set-up kernels of a fill.
//
// Orders (Sec. 3):
//  - naive / spiral: the next B points of a fixed sequence (raster order, or
//    the spiral frames each drawn in random order, Algorithm "spiral
//    method") that are not filled at the start of the round;
//  - minimum filling rate (Algorithm "method based on the filling rate"):
//    the B unfilled points with the smallest fill count cnt, ties going to
//    the greatest geodesic extremum, i.e. the smallest position in the
//    extrema list Ext (Sec. 3.3). With B = 1 this is the paper's loop;
//  - geodesic extrema (Algorithm "geodesic extrema method"): the B unfilled
//    points farthest from the geodesic centroid, ties going to the smallest
//    fill count, then to the smallest index.
// "Filled" is tau(x) = 1, i.e. cnt(x) = N (Sec. 2, eq. "filling rate pt").
#include "common.cuh"
#include "internal.h"

namespace gapsp {

namespace {

// Sequence orders: one warp scans forward from the cursor with ballots.
__global__ void k_select_seq(SelectArgs a) {
    const int lane = threadIdx.x;
    if (*a.done) {
        if (lane == 0) {
            *a.nsel = 0;
            if (a.ncand) *a.ncand = 0;
        }
        return;
    }
    int cursor = *a.cursor, ns = 0;
    while (ns < a.B && cursor < a.nseq) {
        const int idx = cursor + lane;
        const int p = idx < a.nseq ? a.seq[idx] : -1;
        const bool ok = p >= 0 && a.cnt[p] < (uint32_t)a.N;
        const unsigned m = __ballot_sync(FULL, ok);
        const int avail = __popc(m), take = min(avail, a.B - ns);
        const int before = __popc(m & ((1u << lane) - 1u));
        if (ok && before < take) a.sel[ns + before] = p;
        if (take < avail) {
            // stop just after the last taken point
            unsigned mm = m;
            for (int i = 0; i < take - 1; ++i) mm &= mm - 1;
            cursor += __ffs(mm);  // position of the take-th set bit, plus one
        } else {
            cursor += min(32, a.nseq - cursor);
        }
        ns += take;
    }
    // lookahead candidates: within the next KL positions of the sequence
    // after the selection, the first K points that are unfilled now and whose
    // rows are not computed yet (the cursor does not move for them)
    int nc = 0;
    if (a.K > 0) {
        int c2 = cursor;
        const int lim = min(a.nseq, cursor + a.KL);
        while (nc < a.K && c2 < lim) {
            const int idx = c2 + lane;
            const int p = idx < lim ? a.seq[idx] : -1;
            const bool ok = p >= 0 && a.cnt[p] < (uint32_t)a.N && !(a.row_done && a.row_done[p]) &&
                            !(a.row_claim && a.row_claim[p]);
            const unsigned m = __ballot_sync(FULL, ok);
            const int take = min(__popc(m), a.K - nc);
            const int before = __popc(m & ((1u << lane) - 1u));
            if (ok && before < take) {
                a.cand[nc + before] = p;
                if (a.row_claim) a.row_claim[p] = 1;
            }
            nc += take;
            c2 += 32;
        }
    }
    const unsigned long long props = a.stats[S_PROPAGATIONS];
    __syncwarp();
    for (int i = lane; i < ns; i += 32) a.sel_log[props + i] = a.sel[i];
    if (lane == 0) {
        *a.cursor = cursor;
        *a.nsel = ns;
        if (a.ncand) *a.ncand = ns ? nc : 0;
        const unsigned long long rounds = a.stats[S_ROUNDS];
        const unsigned long long cur_new = a.stats[S_NEW] >> 1;
        if (rounds > 0) a.round_new_log[rounds - 1] = cur_new - *a.last_new;
        *a.last_new = cur_new;
        if (ns == 0) {
            *a.done = 1;
        } else {
            a.stats[S_ROUNDS] = rounds + 1;
            a.stats[S_PROPAGATIONS] = props + ns;
        }
    }
}

// Radix selection of the B smallest keys among unfilled points, one block of
// 1024 threads. Keys are distinct and below 2^50 (N <= 2^16, cnt <= 2^16):
//   minimum filling rate:  cnt << 17 | rank
//   geodesic extrema:      grank << 34 | cnt << 17 | p
// where grank counts the free points strictly farther from the centroid, so
// that a smaller grank is a farther point and equal distances share it.
constexpr int SEL_THREADS = 1024;

__device__ __forceinline__ unsigned long long key_of(int order, int N, uint32_t c, int32_t r, int32_t g, int p) {
    if (c >= (uint32_t)N || r < 0) return ~0ull;
    if (order == 3) return ((unsigned long long)g << 34) | ((unsigned long long)c << 17) | (unsigned long long)p;
    return ((unsigned long long)c << 17) | (unsigned long long)r;
}

__device__ __forceinline__ unsigned long long mf_key(const SelectArgs& a, int p) {
    return key_of(a.order, a.N, a.cnt[p], a.rank[p], a.order == 3 ? a.grank[p] : 0, p);
}

// Radix selection, 11 bits a pass from the top bit a key can have: the
// need-th smallest (1-based) of the valid keys keyf(0 .. n-1) (~0 = not a
// key). Every thread of the block calls it with the same arguments.
constexpr int RB = 11, NBIN = 1 << RB;

struct SelScratch {
    unsigned hist[NBIN];
    unsigned wsum[32];
    unsigned long long wlo[32], whi[32];
    unsigned long long prefix;
    int need;
};

template <class KeyF>
__device__ unsigned long long radix_select(KeyF keyf, int n, int need, int top, SelScratch& sc,
                                           unsigned long long prefix0 = 0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long prefix = prefix0;
    if (tid == 0) { sc.need = need; sc.prefix = prefix0; }
    for (int shift = ((top - 1) / RB) * RB; shift >= 0; shift -= RB) {
        for (int i = tid; i < NBIN; i += SEL_THREADS) sc.hist[i] = 0;
        __syncthreads();
        // keys sharing a digit within a warp add to its bin once (most keys
        // share the top digits, which would serialise the atomics)
        for (int p0 = 0; p0 < n; p0 += SEL_THREADS) {
            const int p = p0 + tid;
            const unsigned long long k = p < n ? keyf(p) : ~0ull;
            const bool in = k != ~0ull && (k >> (shift + RB)) == (prefix >> (shift + RB));
            const unsigned dig = in ? (unsigned)((k >> shift) & (NBIN - 1)) : (unsigned)NBIN;
            const unsigned peers = __match_any_sync(FULL, dig);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&sc.hist[dig], (unsigned)__popc(peers));
        }
        __syncthreads();
        // block-wide scan of the bins, two per thread, to find the digit
        // that holds the need-th key
        const unsigned h0 = sc.hist[2 * tid], h1 = sc.hist[2 * tid + 1];
        unsigned v = h0 + h1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) sc.wsum[warp] = v;
        const int nd = sc.need;
        __syncthreads();
        if (warp == 0) {
            unsigned w = sc.wsum[lane];
            unsigned x = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += t;
            }
            sc.wsum[lane] = x - w;  // exclusive
        }
        __syncthreads();
        const unsigned incl = v + sc.wsum[warp], excl = incl - h0 - h1;
        if (excl < (unsigned)nd && (unsigned)nd <= incl) {
            const bool first = excl + h0 >= (unsigned)nd;
            sc.need = nd - (int)(first ? excl : excl + h0);
            sc.prefix = prefix | ((unsigned long long)(2 * tid + (first ? 0 : 1)) << shift);
        }
        __syncthreads();
        prefix = sc.prefix;
    }
    return prefix;
}

// The bits in which the valid keys keyf(0 .. n-1) differ: the radix
// selection then starts at the highest of them (`top` = its position + 1),
// with `prefix0` holding the bits all keys share above the first digit.
template <class KeyF>
__device__ void key_span(KeyF keyf, int n, SelScratch& sc, int& top, unsigned long long& prefix0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long lo = ~0ull, hi = 0;
    for (int i = tid; i < n; i += SEL_THREADS) {
        const unsigned long long k = keyf(i);
        if (k != ~0ull) {
            lo = min(lo, k);
            hi = max(hi, k);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(FULL, lo, o));
        hi = max(hi, __shfl_xor_sync(FULL, hi, o));
    }
    if (lane == 0) { sc.wlo[warp] = lo; sc.whi[warp] = hi; }
    __syncthreads();
    lo = sc.wlo[lane];
    hi = sc.whi[lane];
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(FULL, lo, o));
        hi = max(hi, __shfl_xor_sync(FULL, hi, o));
    }
    __syncthreads();  // wlo / whi are free again
    if (lo > hi) {  // no valid key
        top = 1;
        prefix0 = 0;
        return;
    }
    const unsigned long long diff = lo ^ hi;
    top = diff ? 64 - __clzll((long long)diff) : 1;
    const int first = ((top - 1) / RB) * RB + RB;  // bits below this are selected digit by digit
    prefix0 = first >= 64 ? 0 : (lo & ~((1ull << first) - 1ull));
}

// The end of a minfill / extrema selection, once the keys of a window at
// the front of the ranking (at least the (B + KL) smallest, at most WIN)
// are gathered in s_keys / s_pix (s_count of them): the B selected in key
// order, and the lookahead candidates (the K smallest keys of the window
// after the selection whose rows are neither computed nor claimed).
constexpr int WIN = 2048;

// Exclusive prefix sum over the block of one value per thread; `total`
// receives the sum. Every thread calls it.
__device__ __forceinline__ int block_excl_scan(int v, SelScratch& sc, int& total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sc.wsum[warp] = (unsigned)x;
    __syncthreads();
    if (warp == 0) {
        const int w = (int)sc.wsum[lane];
        int y = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += t;
        }
        sc.wsum[lane] = (unsigned)(y - w);
        if (lane == 31) sc.need = y;
    }
    __syncthreads();
    const int r = (int)sc.wsum[warp] + x - v;
    total = sc.need;
    __syncthreads();  // wsum / need are free again
    return r;
}

__device__ void finish_selection(const SelectArgs& a, int want, int top, SelScratch& sc, int& s_count,
                                 unsigned long long* s_keys, int* s_pix, unsigned long long* s_selk, int* s_selp,
                                 int& s_nsel, int& s_ncand, bool have_t1 = false,
                                 unsigned long long t1_known = 0) {
    __shared__ unsigned long long s_ck[WIN];  // candidate keys (~0: not a candidate)
    const int tid = threadIdx.x, lane = tid & 31;
    const int nall = min(s_count, WIN);
    // the radix selections below start at the highest bit in which the
    // window's keys differ
    unsigned long long prefix0 = 0;
    key_span([&](int i) -> unsigned long long { return s_keys[i]; }, nall, sc, top, prefix0);
    // the selection: the `want` smallest keys of the window, in key order
    unsigned long long t1 = ~0ull - 1;
    if (have_t1) t1 = t1_known;
    else if (want > 0 && want < nall)
        t1 = radix_select([&](int i) -> unsigned long long { return s_keys[i]; }, nall, want, top, sc, prefix0);
    // candidates: after the selection, points whose rows are not computed
    // yet; when there are more than K, the K smallest keys among them
    int ncnd = 0;
    if (a.cand) {
        for (int e = tid; e < nall; e += SEL_THREADS) {
            const int p = s_pix[e];
            const bool taken = (a.row_done && a.row_done[p]) || (a.row_claim && a.row_claim[p]);
            const bool c = s_keys[e] > t1 && !taken;
            s_ck[e] = c ? s_keys[e] : ~0ull;
            ncnd += c;
        }
    }
    unsigned long long tk = ~0ull - 1;
    if (a.cand) {
        for (int o = 16; o > 0; o >>= 1) ncnd += __shfl_down_sync(FULL, ncnd, o);
        if (lane == 0 && ncnd) atomicAdd(&s_ncand, ncnd);
        __syncthreads();
        const int nc = s_ncand;
        __syncthreads();
        if (tid == 0) s_ncand = 0;
        if (nc > a.K)
            tk = radix_select([&](int i) -> unsigned long long { return s_ck[i]; }, nall, a.K, top, sc, prefix0);
        __syncthreads();
    }
    for (int e0 = 0; e0 < nall; e0 += SEL_THREADS) {
        const int e = e0 + tid;
        const bool in_sel = e < nall && s_keys[e] <= t1;
        const bool in_cand = e < nall && a.cand && s_ck[e] <= tk;
        const unsigned ms = __ballot_sync(FULL, in_sel), mc = __ballot_sync(FULL, in_cand);
        int bs = 0, bc = 0;
        if (lane == 0) {
            if (ms) bs = atomicAdd(&s_nsel, __popc(ms));
            if (mc) bc = atomicAdd(&s_ncand, __popc(mc));
        }
        bs = __shfl_sync(FULL, bs, 0);
        bc = __shfl_sync(FULL, bc, 0);
        const unsigned below = (1u << lane) - 1u;
        if (in_sel) {
            const int slot = bs + __popc(ms & below);
            if (slot < 1024) {
                s_selk[slot] = s_keys[e];
                s_selp[slot] = s_pix[e];
            }
        }
        if (in_cand) {
            const int slot = bc + __popc(mc & below);
            if (slot < a.K) {
                a.cand[slot] = s_pix[e];
                if (a.row_claim) a.row_claim[s_pix[e]] = 1;
            }
        }
    }
    __syncthreads();
    const int ns = min(s_nsel, want);
    if (tid < ns) {
        const unsigned long long k = s_selk[tid];
        int pos = 0;
        for (int i = 0; i < ns; ++i) pos += s_selk[i] < k;
        a.sel[pos] = s_selp[tid];
        a.sel_log[a.stats[S_PROPAGATIONS] + pos] = s_selp[tid];
    }
    __syncthreads();
    if (tid == 0) {
        *a.nsel = ns;
        if (a.ncand) *a.ncand = ns ? min(s_ncand, a.K) : 0;
        unsigned long long rounds = a.stats[S_ROUNDS];
        unsigned long long cur_new = a.stats[S_NEW] >> 1;
        if (rounds > 0) a.round_new_log[rounds - 1] = cur_new - *a.last_new;
        *a.last_new = cur_new;
        if (ns == 0) {
            *a.done = 1;
        } else {
            a.stats[S_ROUNDS] = rounds + 1;
            a.stats[S_PROPAGATIONS] += ns;
        }
    }
}

// Minfill / extrema selection, one block. Keys order first by a leading field v (cnt for minfill, grank for extrema)
// that never decreases for a point, and the unfilled set only shrinks, so
// the least v among the unfilled points never decreases from round to round
// (a.vfloor keeps last round's). One pass computes the keys, packs the
// unfilled ones (with their point) into shared memory when they fit (CACHE,
// N <= 16384; otherwise later passes read the counts again), and counts
// them by v - vfloor (2048 bins, the last one for everything beyond). When the
// (B + KL)-th smallest key falls in a bin below the last and at most WIN
// keys have a v up to that bin's, those keys are the window the selection
// and the candidates come from (every key with a smaller v is smaller, so
// the B smallest are among them); otherwise the window is the (B + KL)
// smallest keys, found by radix selection over all of them.
template <int ORDER>
__device__ __forceinline__ unsigned long long packed_key(unsigned long long k, int p) {
    // extrema keys end with the point already; minfill keys get it below them
    return ORDER == 3 ? k : ((k << 16) | (unsigned)p);
}
template <int ORDER>
__device__ __forceinline__ unsigned long long unpack_key(unsigned long long pk) {
    return ORDER == 3 ? pk : (pk >> 16);
}
template <int ORDER>
__device__ __forceinline__ int unpack_point(unsigned long long pk) {
    return ORDER == 3 ? (int)(pk & 0x1FFFFull) : (int)(pk & 0xFFFFull);
}
template <int ORDER>
__device__ __forceinline__ uint32_t lead_field(unsigned long long k) {
    return ORDER == 3 ? (uint32_t)(k >> 34) : (uint32_t)(k >> 17);
}

template <int ORDER, bool CACHE>
__global__ void __launch_bounds__(SEL_THREADS) k_select_small(SelectArgs a) {
    extern __shared__ unsigned long long spk[];  // CACHE: packed keys of the unfilled points
    __shared__ SelScratch sc;
    __shared__ int s_count, s_nsel, s_ncand;
    __shared__ unsigned s_vmin;
    __shared__ int s_below;  // some v below the floor: take the general path
    __shared__ int s_bsel, s_below_sel, s_nt;
    __shared__ unsigned long long s_t1, s_tie[256];
    __shared__ unsigned long long s_keys[WIN], s_selk[1024];
    __shared__ int s_pix[WIN], s_selp[1024];
    const int tid = threadIdx.x, lane = tid & 31;
    if (*a.done) {
        if (tid == 0) {
            *a.nsel = 0;
            if (a.ncand) *a.ncand = 0;
        }
        return;
    }
    const uint32_t vfloor = *a.vfloor;
    if (tid == 0) { s_count = 0; s_nsel = 0; s_ncand = 0; s_vmin = 0xFFFFFFFFu; s_below = 0; }
    for (int i = tid; i < NBIN; i += SEL_THREADS) sc.hist[i] = 0;
    __syncthreads();
    // pass 1, LD points per thread at a time: their counts and ranks are
    // loaded before any is used (the latencies overlap); the unfilled ones
    // are packed in order of a block-wide prefix sum (no shared counter) and
    // binned by v - vfloor.
    constexpr int LD = 8;
    unsigned vmin = 0xFFFFFFFFu;
    int unfilled = 0;
    for (int b0 = 0; b0 < a.N; b0 += LD * SEL_THREADS) {
        uint32_t cv[LD];
        int32_t rv[LD], gv[LD];
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int q = b0 + u * SEL_THREADS + tid;
            cv[u] = (uint32_t)a.N;
            rv[u] = -1;
            gv[u] = 0;
            if (q < a.N) {
                cv[u] = __ldcg(a.cnt + q);
                rv[u] = __ldg(a.rank + q);
                if (ORDER == 3) gv[u] = __ldg(a.grank + q);
            }
        }
        int nv = 0;
#pragma unroll
        for (int u = 0; u < LD; ++u) nv += cv[u] < (uint32_t)a.N && rv[u] >= 0;
        int total;
        int w = unfilled + block_excl_scan(nv, sc, total);
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int q = b0 + u * SEL_THREADS + tid;
            const unsigned long long k = q < a.N ? key_of(ORDER, a.N, cv[u], rv[u], gv[u], q) : ~0ull;
            const bool in = k != ~0ull;
            unsigned dig = (unsigned)(NBIN - 1);
            if (in) {
                if (CACHE) spk[w++] = packed_key<ORDER>(k, q);
                const uint32_t v = lead_field<ORDER>(k);
                vmin = min(vmin, v);
                if (v < vfloor) s_below = 1;  // not expected: the floor never passes a key
                dig = v < vfloor ? (unsigned)(NBIN - 1) : min(v - vfloor, (uint32_t)(NBIN - 1));
            }
            // the last bin is not counted: only the bins below it are
            // searched, and few keys share one of them
            if (dig < (unsigned)(NBIN - 1)) atomicAdd(&sc.hist[dig], 1u);
        }
        unfilled += total;
    }
    for (int o = 16; o > 0; o >>= 1) vmin = min(vmin, __shfl_down_sync(FULL, vmin, o));
    if (lane == 0 && vmin != 0xFFFFFFFFu) atomicMin(&s_vmin, vmin);
    __syncthreads();
    const int want = min(unfilled, a.B);
    const int wantc = min(unfilled, a.B + (a.K > 0 ? a.KL : 0));
    if (tid == 0 && s_vmin != 0xFFFFFFFFu) *a.vfloor = s_vmin;
    int top = ORDER == 3 ? 34 : 17;
    for (int n = a.N - 1; n > 0; n >>= 1) ++top;
    // the bins that hold the wantc-th and the want-th key (the last bin when
    // beyond the counted ones), how many keys lie up to the first and below
    // the second
    int bstar = NBIN - 1, bsel = NBIN - 1;
    unsigned upto = 0, below_sel = 0;
    if (tid == 0) { sc.need = NBIN - 1; s_bsel = NBIN - 1; }
    if (wantc > 0) {
        const unsigned h0 = sc.hist[2 * tid], h1 = sc.hist[2 * tid + 1];
        unsigned v = h0 + h1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) sc.wsum[tid >> 5] = v;
        __syncthreads();
        if (tid < 32) {
            const unsigned w0 = sc.wsum[lane];
            unsigned x = w0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += t;
            }
            sc.wsum[lane] = x - w0;
        }
        __syncthreads();
        const unsigned incl = v + sc.wsum[tid >> 5], excl = incl - h0 - h1;
        if (excl < (unsigned)wantc && (unsigned)wantc <= incl) {
            const bool first = excl + h0 >= (unsigned)wantc;
            sc.need = first ? 2 * tid : 2 * tid + 1;
            sc.prefix = first ? excl + h0 : incl;
        }
        if (excl < (unsigned)want && (unsigned)want <= incl) {
            const bool first = excl + h0 >= (unsigned)want;
            s_bsel = first ? 2 * tid : 2 * tid + 1;
            s_below_sel = first ? excl : excl + h0;
        }
        __syncthreads();
        bstar = sc.need;
        upto = (unsigned)sc.prefix;
        bsel = s_bsel;
        below_sel = (unsigned)s_below_sel;
        __syncthreads();
    }
    bool have_t1 = false;
    unsigned long long t1 = ~0ull - 1;
    if (wantc > 0 && !s_below && bstar < NBIN - 1 && upto <= (unsigned)WIN) {
        // the window: every key whose v is at most that bin's (the
        // (B + KL)-th key among them), gathered in one pass
        const uint32_t vmax = vfloor + (uint32_t)bstar;
        auto gather = [&](bool take, unsigned long long k, int p) {
            const unsigned m = __ballot_sync(FULL, take);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&s_count, __popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (take) {
                const int slot = base + __popc(m & ((1u << lane) - 1u));
                s_keys[slot] = k;
                s_pix[slot] = p;
            }
        };
        if (CACHE) {
            for (int i0 = 0; i0 < unfilled; i0 += SEL_THREADS) {
                const int i = i0 + tid;
                const unsigned long long pk = i < unfilled ? spk[i] : ~0ull;
                const bool take = i < unfilled && lead_field<ORDER>(unpack_key<ORDER>(pk)) <= vmax;
                gather(take, unpack_key<ORDER>(pk), unpack_point<ORDER>(pk));
            }
        } else {
            // the keys again from the counts, LD points per thread at a time
            for (int b0 = 0; b0 < a.N; b0 += LD * SEL_THREADS) {
                uint32_t cv[LD];
                int32_t rv[LD], gv[LD];
#pragma unroll
                for (int u = 0; u < LD; ++u) {
                    const int q = b0 + u * SEL_THREADS + tid;
                    cv[u] = (uint32_t)a.N;
                    rv[u] = -1;
                    gv[u] = 0;
                    if (q < a.N) {
                        cv[u] = __ldcg(a.cnt + q);
                        rv[u] = __ldg(a.rank + q);
                        if (ORDER == 3) gv[u] = __ldg(a.grank + q);
                    }
                }
#pragma unroll
                for (int u = 0; u < LD; ++u) {
                    const int q = b0 + u * SEL_THREADS + tid;
                    const unsigned long long k = q < a.N ? key_of(ORDER, a.N, cv[u], rv[u], gv[u], q) : ~0ull;
                    gather(k != ~0ull && lead_field<ORDER>(k) <= vmax, k, q);
                }
            }
        }
        __syncthreads();
        const int ng = s_count;
        if (want > 0 && want < ng && bsel < NBIN - 1) {
            // the want-th key: keys of smaller v are selected, and among
            // those of its own v (few) it has rank want - below_sel
            const uint32_t vsel = vfloor + (uint32_t)bsel;
            if (tid == 0) { s_nt = 0; s_t1 = ~0ull - 1; }
            __syncthreads();
            for (int e = tid; e < ng; e += SEL_THREADS)
                if (lead_field<ORDER>(s_keys[e]) == vsel) {
                    const int slot = atomicAdd(&s_nt, 1);
                    if (slot < 256) s_tie[slot] = s_keys[e];
                }
            __syncthreads();
            const int nt = s_nt;
            if (nt <= 256) {
                if (tid < nt) {
                    const unsigned long long k = s_tie[tid];
                    int r = 0;
                    for (int i = 0; i < nt; ++i) r += s_tie[i] < k;
                    if (r == want - (int)below_sel - 1) s_t1 = k;
                }
                __syncthreads();
                t1 = s_t1;
                have_t1 = true;
            }
        }
    } else if (want > 0) {
        // the window: the (B + KL) smallest keys, by radix selection over
        // all of them
        // (over the cache, or over the counts again at every pass)
        const int n = CACHE ? unfilled : a.N;
        auto keyf = [&](int i) -> unsigned long long {
            return CACHE ? unpack_key<ORDER>(spk[i]) : mf_key(a, i);
        };
        unsigned long long thr = ~0ull - 1;
        if (wantc < unfilled) thr = radix_select(keyf, n, wantc, top, sc);
        for (int i0 = 0; i0 < n; i0 += SEL_THREADS) {
            const int i = i0 + tid;
            const unsigned long long k = i < n ? keyf(i) : ~0ull;
            const bool take = k != ~0ull && k <= thr;
            const unsigned m = __ballot_sync(FULL, take);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&s_count, __popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (take) {
                const int slot = base + __popc(m & ((1u << lane) - 1u));
                if (slot < WIN) { s_keys[slot] = k; s_pix[slot] = CACHE ? unpack_point<ORDER>(spk[i]) : i; }
            }
        }
    }
    __syncthreads();
    finish_selection(a, want, top, sc, s_count, s_keys, s_pix, s_selk, s_selp, s_nsel, s_ncand, have_t1, t1);
}

// Spiral method with repulsion (Algorithm "spiral method with repulsion",
// h = 3), one warp. S is the current turn's list of points not yet filled,
// one bit per ring position (a turn has at most 1020 points: 32 words, one
// per lane). A source is drawn uniformly from S with SplitMix64 (Steele, Lea
// & Flood, OOPSLA 2014); it and its two neighbours on each side of the turn
// (wrapping around on a closed ring) leave S. Filled points leave S at the
// start of each round; an empty S restarts at the outermost turn that has a
// point not yet filled (and not drawn in this round).
__device__ __forceinline__ unsigned long long splitmix_next(unsigned long long& st) {
    unsigned long long z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_select_rep(SelectArgs a, RepArgs r) {
    const int lane = threadIdx.x;
    if (*a.done) { if (lane == 0) *a.nsel = 0; return; }
    RepState st = *r.state;
    unsigned word = r.inS[lane];
    auto warp_sum = [](int v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        return v;
    };
    // points filled by the previous round leave S
    if (st.cur >= 0) {
        const int base = r.fstart[st.cur], len = r.fstart[st.cur + 1] - base;
        for (int b = 0; b < 32; ++b) {
            const int i = lane * 32 + b;
            if (i < len && ((word >> b) & 1u) && a.cnt[r.ring[base + i]] >= (uint32_t)a.N) word &= ~(1u << b);
        }
    }
    int ns = 0;
    while (ns < a.B) {
        int size = warp_sum(__popc(word));
        if (size == 0) {
            st.cur = -1;
            for (int k = 0; k < st.nframes && st.cur < 0; ++k) {
                const int base = r.fstart[k], len = r.fstart[k + 1] - base;
                bool any = false;
                for (int i = lane; i < len; i += 32) {
                    const int p = r.ring[base + i];
                    any |= a.cnt[p] < (uint32_t)a.N && !r.taken[p];
                }
                if (__any_sync(FULL, any)) st.cur = k;
            }
            if (st.cur < 0) break;
            const int base = r.fstart[st.cur], len = r.fstart[st.cur + 1] - base;
            word = 0;
            for (int b = 0; b < 32; ++b) {
                const int i = lane * 32 + b;
                if (i < len) {
                    const int p = r.ring[base + i];
                    if (a.cnt[p] < (uint32_t)a.N && !r.taken[p]) word |= 1u << b;
                }
            }
            size = warp_sum(__popc(word));
        }
        const int base = r.fstart[st.cur], len = r.fstart[st.cur + 1] - base;
        const int jth = (int)(splitmix_next(st.rng) % (unsigned long long)size);  // same on every lane
        // the lane holding the jth point of S, by an exclusive scan of counts
        const int pc = __popc(word);
        int incl = pc;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - pc;
        const bool mine = excl <= jth && jth < incl;
        int at = mine ? lane * 32 + (int)__fns(word, 0, jth - excl + 1) : 0;
        const unsigned who = __ballot_sync(FULL, mine);
        at = __shfl_sync(FULL, at, __ffs(who) - 1);
        const int s = r.ring[base + at];
        if (lane == 0) {
            a.sel[ns] = s;
            r.taken[s] = 1;
        }
        ++ns;
        for (int d = -2; d <= 2; ++d) {
            int i = at + d;
            if (r.fcyc[st.cur]) i = ((i % len) + len) % len;
            if (i >= 0 && i < len && (i >> 5) == lane) word &= ~(1u << (i & 31));
        }
        __syncwarp();
    }
    r.inS[lane] = word;
    const unsigned long long props = a.stats[S_PROPAGATIONS];
    __syncwarp();
    for (int i = lane; i < ns; i += 32) {
        a.sel_log[props + i] = a.sel[i];
        r.taken[a.sel[i]] = 0;
    }
    if (lane == 0) {
        *r.state = st;
        *a.nsel = ns;
        const unsigned long long rounds = a.stats[S_ROUNDS];
        const unsigned long long cur_new = a.stats[S_NEW] >> 1;
        if (rounds > 0) a.round_new_log[rounds - 1] = cur_new - *a.last_new;
        *a.last_new = cur_new;
        if (ns == 0) {
            *a.done = 1;
        } else {
            a.stats[S_ROUNDS] = rounds + 1;
            a.stats[S_PROPAGATIONS] = props + ns;
        }
    }
}

// Fill counts at the start (Sec. 2: D_mrk(i,i) = 1; pairs no path joins are
// known at once) and the zero diagonal of D.
__global__ void k_init(InitArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.N) return;
    uint32_t c = 1;
    if (a.comp) {
        const int l = a.comp[p];
        c = l < 0 ? (uint32_t)a.N : 1u + (uint32_t)(a.N - a.comp_size[l]);
    }
    a.cnt[p] = c;
    a.D[(size_t)p * a.N + p] = 0;
}

// Geodesic centroid per component: argmax of the distance from the boundary,
// ties to the smallest index (Sec. 3.3).
__global__ void k_centroid_max(ExtremaArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.N) return;
    if (a.freef && !a.freef[p]) return;
    const int l = a.comp ? a.comp[p] : 0;
    const unsigned long long key = ((unsigned long long)a.e[p] << 32) | (0xFFFFFFFFull - (unsigned)p);
    atomicMax(a.best + l, key);
}

__global__ void k_centroid_mark(ExtremaArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.N) return;
    const bool rep = a.comp ? (a.comp[p] == p) : (p == 0);
    if (!rep) return;
    const unsigned long long k = a.best[a.comp ? p : 0];
    const int c = (int)(0xFFFFFFFFull - (k & 0xFFFFFFFFull));
    if (c >= 0 && c < a.N) a.cen_flags[c] = 1;
}

// The same ranks by sorting, for N <= 16384 (one block): the keys
// (~g, p) of the free pixels are bitonic-sorted in shared memory; a pixel's
// rank is its position, and the number of free pixels strictly farther from
// the centroid is the position where its run of equal distances starts.
constexpr int RANK_THREADS = 1024;

__global__ void __launch_bounds__(RANK_THREADS) k_rank_sort(ExtremaArgs a) {
    extern __shared__ unsigned long long rk[];
    __shared__ int s_wmax[RANK_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int n2 = 1;
    while (n2 < a.N) n2 <<= 1;
    for (int i = tid; i < n2; i += RANK_THREADS) {
        unsigned long long k = ~0ull;
        if (i < a.N) {
            a.rank[i] = -1;
            a.grank[i] = -1;
            if (!a.freef || a.freef[i]) k = ((unsigned long long)(~a.g[i]) << 32) | (unsigned)i;
        }
        rk[i] = k;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n2; i += RANK_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = rk[i], y = rk[ixj];
                    if ((x > y) == ((i & k) == 0)) {
                        rk[i] = y;
                        rk[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    // each thread owns a contiguous block of positions: run starts, then a
    // block-wide max-scan of them
    const int per = (n2 + RANK_THREADS - 1) / RANK_THREADS;
    const int i0 = tid * per, i1 = min(i0 + per, n2);
    int run = -1;
    for (int i = i0; i < i1; ++i)
        if (rk[i] != ~0ull && (i == 0 || (rk[i - 1] >> 32) != (rk[i] >> 32))) run = i;
    int x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x = max(x, t);
    }
    if (lane == 31) s_wmax[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = s_wmax[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w = max(w, t);
        }
        s_wmax[lane] = w;
    }
    __syncthreads();
    int cur = __shfl_up_sync(FULL, x, 1);  // max over earlier threads of this warp
    if (lane == 0) cur = -1;
    if (warp > 0) cur = max(cur, s_wmax[warp - 1]);
    for (int i = i0; i < i1; ++i) {
        const unsigned long long k = rk[i];
        if (k == ~0ull) break;  // the keys of obstacles and padding come last
        if (i == 0 || (rk[i - 1] >> 32) != (k >> 32)) cur = i;
        const int p = (int)(k & 0xFFFFFFFFu);
        a.rank[p] = i;
        a.grank[p] = cur;
    }
}

// Position in the extrema list Ext: free pixels by decreasing distance from
// the centroid, ties by increasing index; and the number of free pixels
// strictly farther from the centroid. Counted directly.
// Larger images (N > 16384): ranks from sorted chunks. Each block sorts
// 16384 keys (not g, p), padding and obstacles as all ones, in shared memory
// (bitonic) and writes them to a.keys; the rank of p is then the number of
// keys below its own over all chunks, and its count of points strictly
// farther from the centroids the number of keys below (not g, 0), each
// found by a binary search in every chunk.
constexpr int RANK_CHUNK = 16384;

__global__ void __launch_bounds__(RANK_THREADS) k_rank_chunks(ExtremaArgs a) {
    extern __shared__ unsigned long long ck[];
    const int tid = threadIdx.x, c0 = blockIdx.x * RANK_CHUNK;
    for (int i = tid; i < RANK_CHUNK; i += RANK_THREADS) {
        const int p = c0 + i;
        unsigned long long k = ~0ull;
        if (p < a.N && (!a.freef || a.freef[p])) k = ((unsigned long long)(~a.g[p]) << 32) | (unsigned)p;
        ck[i] = k;
    }
    __syncthreads();
    for (int k = 2; k <= RANK_CHUNK; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < RANK_CHUNK; i += RANK_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = ck[i], y = ck[ixj];
                    if ((x > y) == ((i & k) == 0)) {
                        ck[i] = y;
                        ck[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = tid; i < RANK_CHUNK; i += RANK_THREADS) a.keys[c0 + i] = ck[i];
}

// Number of keys of the sorted chunk below x.
__device__ __forceinline__ int below(const unsigned long long* chunk, unsigned long long x) {
    int lo = 0, hi = RANK_CHUNK;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (chunk[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_rank_merge(ExtremaArgs a, int chunks) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.N) return;
    if (a.freef && !a.freef[p]) {
        a.rank[p] = -1;
        a.grank[p] = -1;
        return;
    }
    const unsigned long long hi = (unsigned long long)(~a.g[p]) << 32;
    const unsigned long long key = hi | (unsigned)p;
    int r = 0, gr = 0;
    for (int c = 0; c < chunks; ++c) {
        const unsigned long long* chunk = a.keys + (size_t)c * RANK_CHUNK;
        r += below(chunk, key);
        gr += below(chunk, hi);
    }
    a.rank[p] = r;
    a.grank[p] = gr;
}

__global__ void k_rank(ExtremaArgs a) {
    __shared__ uint32_t sg[1024];
    __shared__ uint8_t sf[1024];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool have = p < a.N && (!a.freef || a.freef[p]);
    const uint32_t gp = have ? a.g[p] : 0;
    int r = 0, gr = 0;
    for (int base = 0; base < a.N; base += 1024) {
        __syncthreads();
        for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
            const int q = base + i;
            sg[i] = q < a.N ? a.g[q] : 0;
            sf[i] = q < a.N && (!a.freef || a.freef[q]);
        }
        __syncthreads();
        if (have) {
            const int lim = min(1024, a.N - base);
            for (int i = 0; i < lim; ++i) {
                const int q = base + i;
                r += sf[i] && (sg[i] > gp || (sg[i] == gp && q < p));
                gr += sf[i] && sg[i] > gp;
            }
        }
    }
    if (p < a.N) {
        a.rank[p] = have ? r : -1;
        a.grank[p] = have ? gr : -1;
    }
}

// Connected components of free pixels by minimum-label propagation with
// pointer jumping, in one block; the label is the smallest pixel index of
// the component.
__global__ void k_components(CompArgs a) {
    __shared__ int s_changed;
    const int N = a.H * a.W;
    for (int p = threadIdx.x; p < N; p += blockDim.x) a.label[p] = a.freef[p] ? p : -1;
    __syncthreads();
    for (int iter = 0; iter <= N + 1; ++iter) {
        if (threadIdx.x == 0) s_changed = 0;
        __syncthreads();
        int ch = 0;
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            int l = a.label[p];
            if (l < 0) continue;
            const int r = p / a.W, c = p - r * a.W;
            int m = l;
            for (int dr = -1; dr <= 1; ++dr)
                for (int dc = -1; dc <= 1; ++dc) {
                    if (!dr && !dc) continue;
                    if (a.conn == 4 && dr && dc) continue;
                    const int rr = r + dr, cc = c + dc;
                    if (rr < 0 || rr >= a.H || cc < 0 || cc >= a.W) continue;
                    const int lq = ((volatile int*)a.label)[rr * a.W + cc];
                    if (lq >= 0 && lq < m) m = lq;
                }
            m = min(m, ((volatile int*)a.label)[m]);
            if (m < l) { a.label[p] = m; ch = 1; }
        }
        if (ch) s_changed = 1;
        __syncthreads();
        if (!s_changed) break;
        if (iter == N + 1 && threadIdx.x == 0) atomicOr(a.status, ST_NOT_CONVERGED);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < N; p += blockDim.x) a.size[p] = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < N; p += blockDim.x)
        if (a.label[p] >= 0) atomicAdd(a.size + a.label[p], 1);
}

}  // namespace

cudaError_t launch_select(const SelectArgs& a, cudaStream_t st) {
    if (a.order == 2 || a.order == 3) {
        if (a.N <= 16384) {
            static std::atomic<unsigned long long> attr{0};
            once_per_device(attr, [] {
                cudaFuncSetAttribute(k_select_small<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8);
                cudaFuncSetAttribute(k_select_small<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8);
            });
            if (a.order == 2) k_select_small<2, true><<<1, SEL_THREADS, (size_t)a.N * 8, st>>>(a);
            else k_select_small<3, true><<<1, SEL_THREADS, (size_t)a.N * 8, st>>>(a);
        } else {
            // the keys do not fit in shared memory: read from the counts
            if (a.order == 2) k_select_small<2, false><<<1, SEL_THREADS, 0, st>>>(a);
            else k_select_small<3, false><<<1, SEL_THREADS, 0, st>>>(a);
        }
    }
    else k_select_seq<<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_select_repulsion(const SelectArgs& a, const RepArgs& r, cudaStream_t st) {
    k_select_rep<<<1, 32, 0, st>>>(a, r);
    return cudaGetLastError();
}

cudaError_t launch_init(const InitArgs& a, cudaStream_t st) {
    if (a.full_init) {
        cudaError_t e = cudaMemsetAsync(a.D, 0xFF, (size_t)a.N * a.N * sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
    }
    k_init<<<(a.N + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_centroids(const ExtremaArgs& a, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.best, 0, (size_t)a.N * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.cen_flags, 0, (size_t)a.N, st);
    if (e != cudaSuccess) return e;
    k_centroid_max<<<(a.N + 255) / 256, 256, 0, st>>>(a);
    k_centroid_mark<<<(a.N + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rank(const ExtremaArgs& a, cudaStream_t st) {
    if (a.N <= 16384) {
        static std::atomic<unsigned long long> attr{0};
        once_per_device(attr, [] {
            cudaFuncSetAttribute(k_rank_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8);
        });
        int n2 = 1;
        while (n2 < a.N) n2 <<= 1;
        k_rank_sort<<<1, RANK_THREADS, (size_t)n2 * 8, st>>>(a);
    } else if (a.keys) {
        static std::atomic<unsigned long long> attr2{0};
        once_per_device(attr2, [] {
            cudaFuncSetAttribute(k_rank_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, RANK_CHUNK * 8);
        });
        const int chunks = (a.N + RANK_CHUNK - 1) / RANK_CHUNK;
        k_rank_chunks<<<chunks, RANK_THREADS, (size_t)RANK_CHUNK * 8, st>>>(a);
        k_rank_merge<<<(a.N + 255) / 256, 256, 0, st>>>(a, chunks);
    } else {
        k_rank<<<(a.N + 255) / 256, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_components(const CompArgs& a, cudaStream_t st) {
    k_components<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gapsp
