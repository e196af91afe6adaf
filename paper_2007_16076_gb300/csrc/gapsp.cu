// Host runtime and C ABI of gapsp (declared in include/gapsp.h).
//
// A handle owns the device copy of one image and everything a fill needs:
// the fill counts, the tiled marks, the selected sources, the per-source
// trees and the counters. The round loop is driven from the host: each
// round launches selection (c), propagation (a), parents and segments (a')
// and the fill (b) on the handle's stream; every kernel of a round reads
// the device-side selection count and does nothing once the loop is over,
// so rounds are enqueued in chunks and the host only checks the device
// "done" flag between chunks.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gapsp.h"
#include "common.cuh"
#include "internal.h"
#include "runtime.h"

using namespace gapsp;


bool gapsp::is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

namespace gapsp {
namespace rt {

// Host-side fault injection (gapsp_debug_fail_alloc): allocations left
// before one fails; negative = never.
std::atomic<int> g_fail_after{-1};
// Device and pinned host allocations the library holds (gapsp_debug_fail_alloc).
std::atomic<long long> g_live{0};

bool injected_failure() {
    int n = g_fail_after.load();
    while (n >= 0) {
        if (g_fail_after.compare_exchange_weak(n, n - 1)) return n == 0;
    }
    return false;
}

// Pinned host words for the asynchronous copies of a fill's "done" flags
// and status words: one process-wide pinned array handed out kWords at a
// time, allocated once and never freed (allocating and freeing pinned
// memory synchronises the device).
struct PinnedSlots {
    static constexpr int kSlots = 4096, kWords = 4;
    std::mutex mu;
    int* base = nullptr;
    std::vector<int> free_list;
};
PinnedSlots g_pinned;

cudaError_t halloc(int** p) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    std::lock_guard<std::mutex> lock(g_pinned.mu);
    if (!g_pinned.base) {
        const cudaError_t e = cudaMallocHost((void**)&g_pinned.base,
                                             sizeof(int) * PinnedSlots::kSlots * PinnedSlots::kWords);
        if (e != cudaSuccess) {
            g_pinned.base = nullptr;
            return e;
        }
        for (int i = PinnedSlots::kSlots - 1; i >= 0; --i) g_pinned.free_list.push_back(i);
    }
    if (g_pinned.free_list.empty()) return cudaErrorMemoryAllocation;
    *p = g_pinned.base + (size_t)g_pinned.free_list.back() * PinnedSlots::kWords;
    g_pinned.free_list.pop_back();
    g_live.fetch_add(1);
    return cudaSuccess;
}

void hfree(int*& p) {
    if (p) {
        std::lock_guard<std::mutex> lock(g_pinned.mu);
        g_pinned.free_list.push_back((int)((p - g_pinned.base) / PinnedSlots::kWords));
        g_live.fetch_sub(1);
    }
    p = nullptr;
}

// Staging buffers for arrays in host memory (up to 17 GB at 256 x 256):
// plain allocations, kept by the handle, so that repeated calls do not grow
// and trim the stream-ordered pool by that much each time.
template <class T>
cudaError_t salloc(T** p, size_t count) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
    if (e == cudaSuccess) g_live.fetch_add(1);
    else *p = nullptr;
    return e;
}

template <class T>
void sfree(T*& p) {
    if (p) {
        cudaFree(p);
        g_live.fetch_sub(1);
    }
    p = nullptr;
}

// Freed blocks up to this size stay in the device's pool for the next
// handle instead of going back to the driver at every synchronisation.
void keep_pool_warm() {
    static std::atomic<unsigned long long> done{0};
    once_per_device(done, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = 1ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
}

// The last failing CUDA runtime call of this host thread, for
// gapsp_last_error_detail.
thread_local char t_detail[256] = "";

void note_cuda_error(cudaError_t e, const char* call, int line) {
    std::snprintf(t_detail, sizeof t_detail, "gapsp.cu:%d: %s: %s", line, call, cudaGetErrorString(e));
}

#define CK(x)                                                  \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) {                               \
            cudaGetLastError();                                \
            note_cuda_error(e_, #x, __LINE__);                 \
            return e_ == cudaErrorMemoryAllocation ? GAPSP_E_NOMEM : GAPSP_E_CUDA; \
        }                                                      \
    } while (0)

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the generator behind the
// spiral order's random draws.
uint64_t splitmix_next(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Spiral order (Sec. 3.1): frames of pixels at equal distance from the
// image border, outermost first; each frame in a uniformly random order
// (Fisher-Yates driven by one SplitMix64 stream per frame). Taking the next
// unfilled point of this sequence draws uniformly among the frame's
// unfilled points, as Algorithm "spiral method" does.
// Turns of the spiral as rings (Sec. 3.2): frame k's free pixels clockwise
// from (k, k); a frame with two rows and two columns or more is closed.
int spiral_rings(int H, int W, const std::vector<uint8_t>& freef, std::vector<int32_t>& ring,
                 std::vector<int32_t>& fstart, std::vector<uint8_t>& fcyc) {
    const int nf = (std::min(H, W) + 1) / 2;
    ring.clear();
    fstart.assign(nf + 1, 0);
    fcyc.assign(nf, 0);
    auto push = [&](int r, int c) {
        const int p = r * W + c;
        if (freef.empty() || freef[p]) ring.push_back(p);
    };
    for (int k = 0; k < nf; ++k) {
        const int r0 = k, r1 = H - 1 - k, c0 = k, c1 = W - 1 - k;
        fstart[k] = (int)ring.size();
        fcyc[k] = (uint8_t)(r1 > r0 && c1 > c0);
        for (int c = c0; c <= c1; ++c) push(r0, c);
        if (r1 > r0) {
            for (int r = r0 + 1; r <= r1; ++r) push(r, c1);
            if (c1 > c0) {
                for (int c = c1 - 1; c >= c0; --c) push(r1, c);
                for (int r = r1 - 1; r > r0; --r) push(r, c0);
            }
        }
    }
    fstart[nf] = (int)ring.size();
    return nf;
}

std::vector<int32_t> spiral_sequence(int H, int W, uint64_t seed, const std::vector<uint8_t>& freef) {
    std::vector<std::vector<int32_t>> frames((std::min(H, W) + 1) / 2);
    for (int p = 0; p < H * W; ++p) {
        if (!freef.empty() && !freef[p]) continue;
        const int r = p / W, c = p % W;
        const int k = std::min(std::min(r, c), std::min(H - 1 - r, W - 1 - c));
        frames[k].push_back(p);
    }
    std::vector<int32_t> out;
    out.reserve(H * W);
    for (size_t k = 0; k < frames.size(); ++k) {
        std::vector<int32_t>& fr = frames[k];
        uint64_t st = seed ^ ((uint64_t)k * 0x9E3779B97F4A7C15ull);
        for (int i = (int)fr.size() - 1; i >= 1; --i) {
            const int j = (int)(splitmix_next(st) % (uint64_t)(i + 1));
            std::swap(fr[i], fr[j]);
        }
        out.insert(out.end(), fr.begin(), fr.end());
    }
    return out;
}

PropArgs base_prop(const gapsp_handle* h) {
    PropArgs a{};
    a.H = h->H;
    a.W = h->W;
    a.N = h->N;
    a.conn = h->conn;
    a.kind_mask = h->kind == GAPSP_MASK;
    a.level_bytes = h->kind == GAPSP_SUM ? 2 : 1;
    a.f = h->f;
    a.status = h->status;
    a.max_sweeps = 4 * (h->max_sweep_rounds ? h->max_sweep_rounds : h->N + 2);
    a.phases = h->sweep_phases ? h->sweep_phases : 4;
    // one block per source unless its map does not fit in one block's shared
    // memory (then the launch splits it into row strips over a cluster);
    // splitting smaller maps costs more rounds than it saves (measured)
    a.cluster = h->prop_blocks ? h->prop_blocks : 1;
    return a;
}

size_t fill_state_bytes(const gapsp_handle* h) {
    const size_t N = h->N, B = h->B;
    // marks; parent, seg, jmp, acc per source; cnt, cnt_base, seq,
    // rank, grank, round_new, sel_log, emap, gmap, best, cen, row_done per
    // point; the lookahead candidate buffers
    return N * h->words * 8 + B * N * (4 + 16 + 8 + 8) +
           N * (4 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 8 + 1 + 1 + 1 + 4 + 4 + 1 + 1) + 2 * 1024 * 4 + 4096 +
           (N <= 16384 ? 4 * kDepRing * B * N : 0);  // trees handed to k_depths
}

void free_fill_state(gapsp_handle* h);

gapsp_status alloc_fill_state(gapsp_handle* h, cudaStream_t st);

// The fill state is allocated on the first all-pairs call (on the stream
// the fill runs on) and kept; a failed allocation frees whatever part of it
// was made.
gapsp_status ensure_fill_state(gapsp_handle* h, cudaStream_t st) {
    if (h->fill_ready) return GAPSP_OK;
    const gapsp_status gs = alloc_fill_state(h, st);
    if (gs != GAPSP_OK) {
        free_fill_state(h);
        return gs;
    }
    h->fill_ready = true;
    return GAPSP_OK;
}

gapsp_status alloc_fill_state(gapsp_handle* h, cudaStream_t st) {
    const size_t N = h->N, B = h->B;
    CK(dalloc(&h->cnt, N, st));
    CK(dalloc(&h->cnt_base, N, st));
    CK(dalloc(&h->marks, N * h->words, st));
    CK(dalloc(&h->parent, B * N, st));
    CK(dalloc(&h->seg, B * N, st));
    CK(dalloc(&h->jmp, 2 * B * N, st));
    CK(dalloc(&h->acc, 2 * B * N, st));
    CK(dalloc(&h->sel, B, st));
    CK(dalloc(&h->nsel, 1, st));
    CK(dalloc(&h->cursor, 1, st));
    CK(dalloc(&h->done, 1, st));
    CK(dalloc(&h->seq, N, st));
    CK(dalloc(&h->rank, N, st));
    CK(dalloc(&h->grank, N, st));
    CK(dalloc(&h->row_done, N, st));
    CK(dalloc(&h->row_claim, N, st));
    CK(dalloc(&h->rp_ring, N, st));
    CK(dalloc(&h->rp_fstart, N + 2, st));
    CK(dalloc(&h->rp_fcyc, N + 1, st));
    CK(dalloc(&h->rp_inS, 32, st));
    CK(dalloc(&h->rp_state, 1, st));
    CK(dalloc(&h->rp_taken, N, st));
    CK(dalloc(&h->cand, 2 * 1024, st));
    CK(dalloc(&h->ncand, 2, st));
    if (N <= 16384) {
        CK(dalloc(&h->dep_exit, kDepRing * B * N, st));
        CK(dalloc(&h->dep_size, kDepRing * B * N, st));
        CK(dalloc(&h->dep_count, kDepRing, st));
    }
    CK(dalloc(&h->stats, S_SLOTS, st));
    CK(dalloc(&h->round_new, N + 1, st));
    CK(dalloc(&h->last_new, 1, st));
    CK(dalloc(&h->vfloor, 1, st));
    CK(dalloc(&h->sel_log, N + 1, st));
    CK(dalloc(&h->emap, N, st));
    CK(dalloc(&h->gmap, N, st));
    CK(dalloc(&h->best, (N + 16383) / 16384 * 16384, st));  // also the rank sort's scratch
    CK(dalloc(&h->cen, N, st));
    CK(halloc(&h->h_done));
    return GAPSP_OK;
}

void free_fill_state(gapsp_handle* h) {
    dfree(h->cnt, h->st); dfree(h->cnt_base, h->st); dfree(h->marks, h->st); dfree(h->parent, h->st); dfree(h->seg, h->st); dfree(h->jmp, h->st); dfree(h->acc, h->st);
    dfree(h->sel, h->st); dfree(h->nsel, h->st); dfree(h->cursor, h->st); dfree(h->done, h->st); dfree(h->seq, h->st); dfree(h->rank, h->st); dfree(h->grank, h->st);
    dfree(h->row_done, h->st); dfree(h->row_claim, h->st); dfree(h->cand, h->st); dfree(h->ncand, h->st);
    dfree(h->rp_ring, h->st); dfree(h->rp_fstart, h->st); dfree(h->rp_fcyc, h->st); dfree(h->rp_inS, h->st); dfree(h->rp_state, h->st);
    dfree(h->rp_taken, h->st);
    dfree(h->dep_exit, h->st); dfree(h->dep_size, h->st); dfree(h->dep_count, h->st);
    dfree(h->stats, h->st); dfree(h->round_new, h->st); dfree(h->last_new, h->st); dfree(h->vfloor, h->st); dfree(h->sel_log, h->st);
    dfree(h->emap, h->st); dfree(h->gmap, h->st); dfree(h->best, h->st); dfree(h->cen, h->st);
    hfree(h->h_done);
    h->fill_ready = false;
}

void free_all(gapsp_handle* h) {
    cudaStream_t st = h->st;
    dfree(h->f, st); dfree(h->pgeo, st); dfree(h->tbase, st); dfree(h->bound, st); dfree(h->comp, st);
    dfree(h->comp_size, st); dfree(h->status, st); dfree(h->changed, st); dfree(h->bad, st);
    free_fill_state(h);
    dfree(h->src_dev, st);
    if (h->Dtmp || h->out_tmp) {
        // the staging buffers of host arrays: after the handle's work
        cudaStreamSynchronize(st);
        sfree(h->Dtmp);
        sfree(h->out_tmp);
    }
    for (auto& t : h->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    h->timed.clear();
    for (auto e : h->pool) cudaEventDestroy(e);
    h->pool.clear();
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    h->ev0 = h->ev1 = nullptr;
}

enum { K_SELECT = 0, K_PROP = 1, K_TREE = 2, K_AHEAD = 3, K_FILL = 4, K_INIT = 5, K_PRE = 6, K_DEPTH = 7,
       K_RECOUNT = 8, K_MIRROR = 9 };

cudaEvent_t pool_get(gapsp_handle* h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch with events when profiling is on.
struct ProfScope {
    gapsp_handle* h;
    bool on;
    ProfScope(gapsp_handle* hh, int kind, cudaStream_t s) : h(hh), on(hh->prof) {
        if (!on) return;
        gapsp_handle::Timed t{kind, pool_get(h), pool_get(h)};
        cudaEventRecord(t.a, s);
        h->timed.push_back(t);
        stream = s;
    }
    ~ProfScope() {
        if (on) cudaEventRecord(h->timed.back().b, stream);
    }
    cudaStream_t stream = nullptr;
};

}  // namespace rt
}  // namespace gapsp

using namespace gapsp::rt;

extern "C" {

void gapsp_default_opts(gapsp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->conn = 8;
    o->kind = GAPSP_GREY;
    o->B = 32;
}

const char* gapsp_strerror(gapsp_status s) {
    switch (s) {
        case GAPSP_OK: return "ok";
        case GAPSP_E_INVALID: return "invalid argument";
        case GAPSP_E_NOMEM: return "out of memory";
        case GAPSP_E_BUDGET: return "memory budget exceeded";
        case GAPSP_E_CUDA: return "CUDA runtime error";
        case GAPSP_E_NOT_CONVERGED: return "propagation did not converge within its sweep limit";
        case GAPSP_E_TIMEOUT: return "round loop exceeded its round limit";
        case GAPSP_E_CANCELLED: return "cancelled";
        case GAPSP_E_CHECK: return "result failed its certificate";
    }
    return "unknown status";
}

uint64_t gapsp_kernel_launches(const gapsp_handle* h) { return h ? h->launches : 0; }

}  // extern "C"

// gapsp_create and gapsp_create_channels: `img` holds L channel planes when
// L > 0 (the GAPSP_SUM kind), else one plane of grey levels or free flags.
static gapsp_status create_handle(const uint8_t* img, int L, int H, int W, const uint8_t* mask,
                                  const gapsp_opts* opts, gapsp_handle** out) {
    if (!out) return GAPSP_E_INVALID;
    *out = nullptr;
    gapsp_opts o;
    gapsp_default_opts(&o);
    if (opts) o = *opts;
    if (L > 0) {
        o.kind = GAPSP_SUM;
        if (L > GAPSP_MAX_CHANNELS) return GAPSP_E_INVALID;
        // every distance must stay below the sweeps' "unreached" sentinel
        if ((long long)(H * W - 1) * (510LL * L + 1) >= (1LL << 30) - (1LL << 18)) return GAPSP_E_INVALID;
    } else if (o.kind == GAPSP_SUM) {
        return GAPSP_E_INVALID;  // needs the channels (gapsp_create_channels)
    }
    if (o.conn == 0) o.conn = 8;
    if (o.B == 0) o.B = 32;
    if (H < 1 || W < 1 || H > GAPSP_MAX_SIDE || W > GAPSP_MAX_SIDE || H * W > GAPSP_MAX_N) return GAPSP_E_INVALID;
    if (o.conn != 4 && o.conn != 8) return GAPSP_E_INVALID;
    if (o.kind != GAPSP_GREY && o.kind != GAPSP_MASK && o.kind != GAPSP_L1 && o.kind != GAPSP_SUM)
        return GAPSP_E_INVALID;
    if (o.B < 1 || o.B > 1024) return GAPSP_E_INVALID;
    if (o.sweep_phases < 0 || o.sweep_phases > 4 || o.sweep_phases == 3) return GAPSP_E_INVALID;
    if (o.fill_rows < -3 || o.fill_rows > 32) return GAPSP_E_INVALID;
    if (o.prop_blocks != 0 && o.prop_blocks != 1 && o.prop_blocks != 2 && o.prop_blocks != 4)
        return GAPSP_E_INVALID;
    if (o.lookahead < -1 || o.lookahead > 1024) return GAPSP_E_INVALID;
    if (o.warm_start != 0 && o.warm_start != -1) return GAPSP_E_INVALID;
    if (o.max_sweep_rounds < 0 || o.max_rounds < 0) return GAPSP_E_INVALID;
    if (o.checked != 0 && o.checked != 1) return GAPSP_E_INVALID;
    if (o.kind != GAPSP_MASK && !img) return GAPSP_E_INVALID;
    if (o.kind == GAPSP_MASK && !mask) return GAPSP_E_INVALID;

    gapsp_handle* h = new (std::nothrow) gapsp_handle();
    if (!h) return GAPSP_E_NOMEM;
    h->H = H; h->W = W; h->N = H * W; h->conn = o.conn; h->kind = o.kind; h->B = o.B;
    h->seed = o.seed; h->budget = o.mem_budget; h->st = (cudaStream_t)o.stream;
    h->sweep_phases = o.sweep_phases;
    h->fill_rows = o.fill_rows;
    h->prop_blocks = o.prop_blocks;
    h->lookahead = o.lookahead;
    h->warm = o.warm_start == 0;
    h->max_sweep_rounds = o.max_sweep_rounds;
    h->max_rounds = o.max_rounds;
    h->checked = o.checked == 1;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            h->sms = 0;
        }
    }
    h->tiles_w = (W + 7) / 8; h->tiles_h = (H + 7) / 8; h->words = h->tiles_w * h->tiles_h;
    const size_t N = h->N;
    if (h->budget && N * 32 + 4096 > h->budget) { delete h; return GAPSP_E_BUDGET; }

    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return e == cudaErrorMemoryAllocation ? GAPSP_E_NOMEM : GAPSP_E_CUDA;
    };
    keep_pool_warm();
    cudaError_t e;
    // levels: one byte per pixel, two for the channel sum
    if ((e = dalloc(&h->f, L > 0 ? 2 * N : N, h->st)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&h->pgeo, N, h->st)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&h->tbase, (size_t)h->words, h->st)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&h->bound, N, h->st)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&h->status, 1, h->st)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&h->changed, 1, h->st)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&h->bad, 1, h->st)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return fail(e);
    // the kernels read grey levels (grey) or free flags (mask) from h->f
    const uint8_t* srcimg = o.kind == GAPSP_MASK ? mask : img;
    if (L > 0) {
        // F = sum of the channels, in 16-bit levels
        uint8_t* planes = nullptr;
        if ((e = dalloc(&planes, (size_t)L * N, h->st)) != cudaSuccess) return fail(e);
        e = cudaMemcpyAsync(planes, img, (size_t)L * N, cudaMemcpyDefault, h->st);
        if (e == cudaSuccess) e = launch_channel_sum(planes, L, (int)N, reinterpret_cast<uint16_t*>(h->f), h->st);
        dfree(planes, h->st);
        if (e != cudaSuccess) return fail(e);
        h->launches += 1;
    } else if ((e = cudaMemcpyAsync(h->f, srcimg, N, cudaMemcpyDefault, h->st)) != cudaSuccess) {
        return fail(e);
    }
    if ((e = cudaMemsetAsync(h->status, 0, sizeof(int), h->st)) != cudaSuccess) return fail(e);
    if (o.kind == GAPSP_MASK) {
        // normalise the flags to 0/1
        std::vector<uint8_t> m(N);
        if ((e = cudaMemcpyAsync(m.data(), mask, N, cudaMemcpyDefault, h->st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(h->st)) != cudaSuccess)
            return fail(e);
        for (auto& v : m) v = v ? 1 : 0;
        if ((e = cudaMemcpyAsync(h->f, m.data(), N, cudaMemcpyHostToDevice, h->st)) != cudaSuccess) return fail(e);
        if ((e = cudaStreamSynchronize(h->st)) != cudaSuccess) return fail(e);
    }
    ImagePrep ip{h->f, H, W, o.conn, (int)o.kind, h->bound, h->pgeo, h->tbase, h->tiles_w, h->words};
    if ((e = launch_image_prep(ip, h->st)) != cudaSuccess) return fail(e);
    h->launches += 2;
    if (o.kind == GAPSP_MASK) {
        if ((e = dalloc(&h->comp, N, h->st)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&h->comp_size, N, h->st)) != cudaSuccess) return fail(e);
        CompArgs ca{H, W, o.conn, h->f, h->comp, h->comp_size, h->changed, h->status};
        if ((e = launch_components(ca, h->st)) != cudaSuccess) return fail(e);
        h->launches += 1;
    }
    int sw = 0;
    if ((e = cudaMemcpyAsync(&sw, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->st)) != cudaSuccess)
        return fail(e);
    if (sw) {
        free_all(h);
        delete h;
        return status_from_word(sw);
    }
    *out = h;
    return GAPSP_OK;
}

extern "C" {

gapsp_status gapsp_create(const uint8_t* img, int H, int W, const uint8_t* mask, const gapsp_opts* opts,
                          gapsp_handle** out) {
    return create_handle(img, 0, H, W, mask, opts, out);
}

gapsp_status gapsp_create_channels(const uint8_t* planes, int L, int H, int W, const gapsp_opts* opts,
                                   gapsp_handle** out) {
    if (out) *out = nullptr;
    if (L < 1 || !planes) return GAPSP_E_INVALID;
    return create_handle(planes, L, H, W, nullptr, opts, out);
}

void gapsp_destroy(gapsp_handle* h) {
    if (!h) return;
    free_all(h);  // stream-ordered: after the work queued on the handle's stream
    delete h;
}

gapsp_status gapsp_rows(gapsp_handle* h, const int32_t* sources, int K, uint32_t* out) {
    if (!h || K < 0) return GAPSP_E_INVALID;
    if (K == 0) return GAPSP_OK;
    if (!sources || !out) return GAPSP_E_INVALID;
    const size_t N = h->N;
    std::vector<int32_t> hs(K);
    CK(cudaMemcpyAsync(hs.data(), sources, K * sizeof(int32_t), cudaMemcpyDefault, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int k = 0; k < K; ++k)
        if (hs[k] < 0 || hs[k] >= h->N) return GAPSP_E_INVALID;
    const bool out_dev = is_device_ptr(out);
    if (out_dev && (reinterpret_cast<uintptr_t>(out) & 15)) return GAPSP_E_INVALID;  // 16-byte row stores
    const size_t out_bytes = (size_t)K * N * sizeof(uint32_t);
    if (h->budget && (out_dev ? 0 : out_bytes) + (size_t)K * 4 > h->budget) return GAPSP_E_BUDGET;
    if (K > h->src_cap) {
        dfree(h->src_dev, h->st);
        h->src_cap = 0;
        CK(dalloc(&h->src_dev, K, h->st));
        h->src_cap = K;
    }
    uint32_t* dout = out;
    if (!out_dev) {
        if (h->out_tmp_bytes < out_bytes) {
            sfree(h->out_tmp);
            h->out_tmp_bytes = 0;
            CK(salloc(&h->out_tmp, (size_t)K * N));
            h->out_tmp_bytes = out_bytes;
        }
        dout = h->out_tmp;
    }
    CK(cudaMemcpyAsync(h->src_dev, hs.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
    PropArgs a = base_prop(h);
    a.map_base = (int*)dout;
    a.sources = h->src_dev;
    a.njobs = K;
    a.convert = h->kind == GAPSP_MASK;
    if (!h->sweep_phases) a.phases = K > 304 ? 1 : 4;  // latency-bound when few sources

    const int wpb = 1;
    {
        ProfScope ps(h, K_PROP, h->st);
        CK(launch_propagate(a, h->conn, h->kind, (K + wpb - 1) / wpb, wpb, h->st));
    }
    h->launches += 1;
    if (h->checked) {
        int sw0 = 0;
        CK(cudaMemcpyAsync(&sw0, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        uint64_t bad = 0;
        if (sw0 == 0) {
            const gapsp_status cs = certify_rows(h, dout, h->src_dev, K, h->st, &bad);
            if (cs != GAPSP_OK) return cs;
        }
        if (bad) {
            std::snprintf(t_detail, sizeof t_detail, "certificate: %llu entries of the rows break the distance equations",
                          (unsigned long long)bad);
            return GAPSP_E_CHECK;
        }
    }
    if (!out_dev) CK(cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, h->st));
    int sw = 0;
    CK(cudaMemcpyAsync(&sw, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return status_from_word(sw);
}

}  // extern "C"

namespace gapsp {
namespace rt {


// Candidates propagated ahead per round: one block (cluster) for each
// multiprocessor the round's own sources leave free, unless set by option.
int lookahead_count(const gapsp_handle* h, const PropArgs& pa, int sm_share) {
    // a map in global memory is the output row itself, which the round's
    // fill may write while a lookahead launch sweeps it: no lookahead then
    if (h->lookahead < 0 || !prop_map_in_smem(pa)) return 0;
    int K = h->lookahead;
    if (K == 0) {
        // the multiprocessors this fill may count on: the whole device, or
        // its share when fills run side by side (batch, server)
        const int per = prop_blocks_per_job(pa);
        const int sms = sm_share > 0 ? std::min(sm_share, h->sms) : h->sms;
        K = sms / per - h->B;
    }
    K = std::min(K, 1024 - h->B);
    return K > 0 ? K : 0;
}

gapsp_status fill_begin(FillRun& r) {
    gapsp_handle* h = r.h;
    const size_t N = h->N;
    r.d_dev = is_device_ptr(r.D);
    // rows of D are stored and read 16 bytes at a time
    if (r.d_dev && (reinterpret_cast<uintptr_t>(r.D) & 15)) return GAPSP_E_INVALID;
    const size_t dbytes = N * N * sizeof(uint32_t);
    const size_t need = fill_state_bytes(h) + (r.d_dev ? 0 : dbytes);
    if (h->budget && need > h->budget) return GAPSP_E_BUDGET;
    gapsp_status gs = ensure_fill_state(h, r.s);
    if (gs != GAPSP_OK) return gs;
    r.Dd = r.D;
    if (!r.d_dev) {
        if (h->Dtmp_bytes < dbytes) {
            sfree(h->Dtmp);
            h->Dtmp_bytes = 0;
            CK(salloc(&h->Dtmp, N * N));
            h->Dtmp_bytes = dbytes;
        }
        r.Dd = h->Dtmp;
    }
    cudaStream_t s = r.s;
    uint32_t* Dd = r.Dd;

    // host-built sequences (naive / spiral) and turns (spiral with repulsion)
    const bool ranked = r.order == GAPSP_MINFILL || r.order == GAPSP_EXTREMA;
    if (r.order == GAPSP_REPULSION) {
        std::vector<uint8_t> freef;
        if (h->kind == GAPSP_MASK) {
            freef.resize(N);
            CK(cudaMemcpyAsync(freef.data(), h->f, N, cudaMemcpyDeviceToHost, r.s));
            CK(cudaStreamSynchronize(r.s));
        }
        std::vector<int32_t> ring, fstart;
        std::vector<uint8_t> fcyc;
        const int nf = spiral_rings(h->H, h->W, freef, ring, fstart, fcyc);
        if (!ring.empty())
            CK(cudaMemcpyAsync(h->rp_ring, ring.data(), ring.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->rp_fstart, fstart.data(), fstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (nf) CK(cudaMemcpyAsync(h->rp_fcyc, fcyc.data(), fcyc.size(), cudaMemcpyHostToDevice, s));
        const RepState rs{h->seed, -1, nf};
        CK(cudaMemcpyAsync(h->rp_state, &rs, sizeof(rs), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(h->rp_inS, 0, 32 * sizeof(unsigned), s));
        CK(cudaMemsetAsync(h->rp_taken, 0, N, s));
        CK(cudaStreamSynchronize(s));  // the host vectors go out of scope
        r.ra = RepArgs{h->rp_ring, h->rp_fstart, h->rp_fcyc, h->rp_inS, h->rp_state, h->rp_taken};
    } else if (!ranked) {
        std::vector<uint8_t> freef;
        if (h->kind == GAPSP_MASK) {
            freef.resize(N);
            CK(cudaMemcpyAsync(freef.data(), h->f, N, cudaMemcpyDeviceToHost, r.s));
            CK(cudaStreamSynchronize(r.s));
        }
        std::vector<int32_t> seq;
        if (r.order == GAPSP_NAIVE) {
            for (int p = 0; p < h->N; ++p)
                if (freef.empty() || freef[p]) seq.push_back(p);
        } else {
            seq = spiral_sequence(h->H, h->W, h->seed, freef);
        }
        r.nseq = (int)seq.size();
        if (r.nseq) CK(cudaMemcpyAsync(h->seq, seq.data(), r.nseq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // the host vector goes out of scope
    }

    CK(cudaEventRecord(h->ev0, s));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(h->stats, 0, S_SLOTS * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->last_new, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->vfloor, 0, sizeof(uint32_t), s));
    CK(cudaMemsetAsync(h->cursor, 0, sizeof(int), s));
    CK(cudaMemsetAsync(h->done, 0, sizeof(int), s));
    CK(cudaMemsetAsync(h->nsel, 0, sizeof(int), s));
    CK(cudaMemsetAsync(h->marks, 0, N * h->words * sizeof(unsigned long long), s));
    // D starts as UNREACH everywhere when a mask may leave pairs unjoined,
    // and when propagations start warm from it
    InitArgs ia{h->N, Dd, h->cnt, h->comp, h->comp_size, h->kind == GAPSP_MASK || h->warm};
    // (the mirror pass tells the missing side of a pair by its UNREACH)
    r.one_side_first = (h->fill_rows == -2 || h->fill_rows == -3) && ia.full_init;
    {
        ProfScope ps(h, K_INIT, s);
        CK(launch_init(ia, s));
    }
    CK(cudaMemcpyAsync(h->cnt_base, h->cnt, N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    h->launches += 1;

    r.prepass = 0;
    if (ranked) {
        // geodesic extrema (Sec. 3.3): distance from the boundary vertices,
        // centroid(s), distance from the centroid(s), rank in Ext
        PropArgs a = base_prop(h);
        a.map_base = (int*)h->emap;
        a.seed_flags = h->bound;
        a.njobs = 1;
        a.convert = 1;
        {
            ProfScope ps(h, K_PROP, s);
            CK(launch_propagate(a, h->conn, h->kind, 1, 1, s));
        }
        // (the centroids' scratch is free again when the ranks are sorted)
        ExtremaArgs ea{h->N, h->kind == GAPSP_MASK ? h->f : nullptr, h->comp, h->emap, h->best, h->cen,
                       h->gmap, h->rank, h->grank, h->N > 16384 ? h->best : nullptr};
        {
            ProfScope ps(h, K_PRE, s);
            CK(launch_centroids(ea, s));
        }
        a.map_base = (int*)h->gmap;
        a.seed_flags = h->cen;
        {
            ProfScope ps(h, K_PROP, s);
            CK(launch_propagate(a, h->conn, h->kind, 1, 1, s));
        }
        {
            ProfScope ps(h, K_PRE, s);
            CK(launch_rank(ea, s));
        }
        h->launches += h->N > 16384 ? 7 : 6;  // the larger images rank in two launches
        r.prepass = 2;
    }

    CK(cudaMemsetAsync(h->row_done, 0, N, s));
    CK(cudaMemsetAsync(h->row_claim, 0, N, s));
    r.sa = SelectArgs{h->N, h->B, (int)r.order, h->cnt, h->rank, h->grank, h->seq, r.nseq, h->cursor, h->sel, h->nsel,
                      h->stats, h->round_new, h->last_new, h->sel_log, h->done};
    r.sa.vfloor = h->vfloor;
    PropArgs& pa = r.pa;
    pa = base_prop(h);
    pa.map_base = (int*)Dd;
    pa.map_row = h->sel;
    pa.sources = h->sel;
    pa.njobs_dev = h->nsel;
    pa.convert = h->kind == GAPSP_MASK;
    pa.sweeps = h->stats + S_SWEEPS;
    pa.row_done = h->row_done;
    if (h->warm) pa.warm_rows = Dd;
    // the repulsion order's draws cannot be foreseen: no lookahead
    r.K = r.order == GAPSP_REPULSION ? 0 : lookahead_count(h, pa, r.sm_share);
    if (r.K > 0) {
        r.sa.K = r.K;
        r.sa.KL = 1024 - h->B;
        r.sa.row_done = h->row_done;
        r.sa.row_claim = h->row_claim;
        r.sa.cand = h->cand;
        r.sa.ncand = h->ncand;
        r.pa_ahead = pa;
        r.pa_ahead.ran = h->stats + S_AHEAD;
        pa.hits = h->stats + S_HITS;
        CK(cudaStreamCreateWithFlags(&r.side[0], cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&r.side[1], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&r.e_sel, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&r.e_ahead[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&r.e_ahead[1], cudaEventDisableTiming));
    }
    TreeArgs& ta = r.ta;
    ta = TreeArgs{};
    ta.H = h->H; ta.W = h->W; ta.N = h->N; ta.conn = h->conn; ta.kind = h->kind;
    ta.tiles_w = h->tiles_w; ta.words = h->words;
    ta.wdiv = h->W == 1 ? 0u : (unsigned)((0x100000000ull + (unsigned)h->W - 1) / (unsigned)h->W);
    ta.f = h->f; ta.D = Dd; ta.sel = h->sel; ta.nsel = h->nsel;
    ta.pgeo = h->pgeo; ta.tbase = h->tbase;
    ta.parent = h->parent; ta.seg = h->seg; ta.jmp = h->jmp; ta.acc = h->acc;
    ta.marks = h->marks; ta.cnt = h->cnt; ta.Dw = Dd; ta.stats = h->stats;
    ta.cnt_base = h->cnt_base;
    {
        const size_t row_bytes = fill_smem_bytes(1, h->words);  // marks + changed flags
        int rpb = (int)((96 * 1024) / row_bytes);
        // 8 rows per block: enough blocks per SM to hide the latency of the
        // tree walks (measured best on the 128x128 workload)
        ta.rows_per_block = rpb < 1 ? 1 : (rpb > 8 ? 8 : rpb);
        if (h->fill_rows) ta.rows_per_block = h->fill_rows;
        if ((size_t)ta.rows_per_block * row_bytes > 200 * 1024) ta.rows_per_block = rpb < 1 ? 1 : rpb;
        if (h->fill_rows == 0 || h->fill_rows == -2) ta.rows_per_block = 0;  // marks claimed in global memory
        if (h->fill_rows == -1 || h->fill_rows == -3) ta.rows_per_block = -1;  // walks in lockstep
    }
    r.rounds = 0;
    r.finished = false;
    r.chunks = r.polled = 0;
    r.t_poll = host_seconds();
    CK(cudaEventCreateWithFlags(&r.chunk_ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&r.chunk_ev[1], cudaEventDisableTiming));
    if (h->dep_exit) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&r.stat, cudaStreamNonBlocking, least));
        for (int i = 0; i < kDepRing; ++i) {
            CK(cudaEventCreateWithFlags(&r.e_tree[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&r.e_depth[i], cudaEventDisableTiming));
        }
    }
    return GAPSP_OK;
}


// Enqueues `chunk` rounds and an asynchronous copy of the "done" flag.
gapsp_status fill_enqueue(FillRun& r, int chunk, bool graph) {
    gapsp_handle* h = r.h;
    cudaStream_t s = r.s;
    // captured into a graph: no per-launch timing events, and the chunk is
    // closed on itself (below)
    const bool prof = h->prof;
    if (graph) h->prof = false;
    struct RestoreProf {
        gapsp_handle* h;
        bool v;
        ~RestoreProf() { h->prof = v; }
    } restore{h, prof};
    for (int i = 0; i < chunk; ++i) {
        // the candidate buffers alternate by round: a round's lookahead
        // launch reads one while the next selection writes the other
        const int par = (r.rounds + i) & 1;
        if (r.K > 0) {
            r.sa.cand = h->cand + par * 1024;
            r.sa.ncand = h->ncand + par;
        }
        const int slot = (r.rounds + i) % kDepRing;
        if (r.stat) {
            // this round hands its trees to the depth sums through the
            // buffer of its slot in a ring of kDepRing, once the launch that
            // read it kDepRing rounds ago is done: the depth sums, on a
            // low-priority stream, have the gaps of several rounds to run in
            r.ta.dep_exit = h->dep_exit + (size_t)slot * h->B * h->N;
            r.ta.dep_size = h->dep_size + (size_t)slot * h->B * h->N;
            r.ta.dep_count = h->dep_count + slot;
            // (in a graph, the launch kDepRing rounds ago belongs to the
            // previous chunk, which ended before this one started)
            if (!graph || i >= kDepRing) CK(cudaStreamWaitEvent(s, r.e_depth[slot], 0));
        }
        {
            ProfScope ps(h, K_SELECT, s);
            if (r.order == GAPSP_REPULSION) CK(launch_select_repulsion(r.sa, r.ra, s));
            else CK(launch_select(r.sa, s));
        }
        if (r.K > 0) {
            // this round's candidates go to the lookahead stream of its
            // parity and start at once, beside the previous round's (the
            // selection never hands out a row already claimed) ...
            CK(cudaEventRecord(r.e_sel, s));
            CK(cudaStreamWaitEvent(r.side[par], r.e_sel, 0));
            r.pa_ahead.sources = h->cand + par * 1024;
            r.pa_ahead.map_row = h->cand + par * 1024;
            r.pa_ahead.njobs_dev = h->ncand + par;
            {
                ProfScope ps(h, K_AHEAD, r.side[par]);
                CK(launch_propagate(r.pa_ahead, h->conn, h->kind, r.K, 1, r.side[par]));
            }
            CK(cudaEventRecord(r.e_ahead[par], r.side[par]));
            h->launches += 1;
            // ... and this round's own propagation waits for the previous
            // round's lookahead, which may have computed its sources
            if (!graph || i >= 1) CK(cudaStreamWaitEvent(s, r.e_ahead[par ^ 1], 0));
        }
        {
            ProfScope ps(h, K_PROP, s);
            CK(launch_propagate(r.pa, h->conn, h->kind, h->B, 1, s));
        }
        // propagation, tree, fill and recount follow each other directly on
        // the stream: each later one is a programmatic dependent launch that
        // may be scheduled while the one before drains
        {
            ProfScope ps(h, K_TREE, s);
            CK(launch_tree(r.ta, h->B, s, true));
        }
        // the first round, when it fills most pairs, writes one side of each
        // (the walks in lockstep: whole runs of entries), and the mirror
        // completes the other side before the next round's propagations read
        // rows of the array
        const bool one_side = r.one_side_first && r.rounds + i == 0;
        {
            ProfScope ps(h, K_FILL, s);
            if (one_side) {
                TreeArgs t1 = r.ta;
                t1.rows_per_block = -1;
                t1.one_side = 1;
                CK(launch_fill(t1, h->B, s, true));
            } else {
                CK(launch_fill(r.ta, h->B, s, true));
            }
        }
        if (one_side) {
            // no propagation of this round's lookahead may write the array
            // meanwhile: only exact distances are there to mirror
            if (r.K > 0) CK(cudaStreamWaitEvent(s, r.e_ahead[par], 0));
            ProfScope ps(h, K_MIRROR, s);
            CK(launch_mirror(r.ta.Dw, h->N, s));
            h->launches += 1;
        }
        {
            ProfScope ps(h, K_RECOUNT, s);
            CK(launch_recount(r.ta, s, true));
        }
        if (r.stat) {
            CK(cudaEventRecord(r.e_tree[slot], s));
            CK(cudaStreamWaitEvent(r.stat, r.e_tree[slot], 0));
            {
                ProfScope ps(h, K_DEPTH, r.stat);
                CK(launch_depths(r.ta, h->B, r.stat));
            }
            CK(cudaEventRecord(r.e_depth[slot], r.stat));
            h->launches += 1;
        }
        h->launches += 5;
    }
    r.rounds += chunk;
    if (graph) {
        // a graph's chunk ends with every side stream joined, and its flags
        // always go to the first slot (the host reads them after the launch)
        if (r.K > 0) {
            CK(cudaStreamWaitEvent(s, r.e_ahead[0], 0));
            CK(cudaStreamWaitEvent(s, r.e_ahead[1], 0));
        }
        if (r.stat)
            for (int k = 0; k < kDepRing; ++k) CK(cudaStreamWaitEvent(s, r.e_depth[k], 0));
        CK(cudaMemcpyAsync(h->h_done, h->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h->h_done + 2, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        return GAPSP_OK;
    }
    const int par = r.chunks & 1;
    r.chunk_rounds[par] = chunk;
    CK(cudaMemcpyAsync(h->h_done + par, h->done, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_done + 2 + par, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(r.chunk_ev[par], s));
    ++r.chunks;
    return GAPSP_OK;
}

// Waits for the oldest chunk not yet waited for and reads its "done" flag
// and the status word. Rounds enqueued after the fill is done return at
// once. A device error (a propagation that hit its sweep limit), the round
// limit and a cancel request end the fill here.
gapsp_status fill_poll(FillRun& r) {
    gapsp_handle* h = r.h;
    const int par = r.polled & 1;
    CK(cudaEventSynchronize(r.chunk_ev[par]));
    ++r.polled;
    // the host time since the previous poll, per round of this chunk: the
    // pace of the rounds, which sets the size of the next chunks
    const double now = host_seconds();
    if (r.chunk_rounds[par] > 0) r.round_s = (now - r.t_poll) / r.chunk_rounds[par];
    r.t_poll = now;
    r.finished = h->h_done[par] != 0;
    const gapsp_status dev = status_from_word(h->h_done[2 + par]);
    if (dev != GAPSP_OK) return dev;
    if (h->cancel.load()) return GAPSP_E_CANCELLED;
    const int cap = h->max_rounds ? h->max_rounds : h->N + 2 + 64;
    if (!r.finished && r.rounds - kChunk >= cap) return GAPSP_E_TIMEOUT;
    return GAPSP_OK;
}

gapsp_status certify_rows(gapsp_handle* h, const uint32_t* D, const int32_t* src, int K, cudaStream_t st,
                          uint64_t* bad) {
    CertifyArgs ca{D, K, src, h->H, h->W, h->N, h->conn, h->kind, h->f, h->bad};
    unsigned long long hb = 0;
    CK(cudaMemsetAsync(h->bad, 0, sizeof(unsigned long long), st));
    CK(launch_certify(ca, st));
    h->launches += 1;
    CK(cudaMemcpyAsync(&hb, h->bad, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *bad = hb;
    return GAPSP_OK;
}

bool fill_chunk_ready(const FillRun& r) {
    return cudaEventQuery(r.chunk_ev[r.polled & 1]) != cudaErrorNotReady;
}

// After an error: waits for everything the fill queued on its streams, so
// that no round still writes the caller's array once the call returns.
void fill_drain(FillRun& r) {
    if (r.s) cudaStreamSynchronize(r.s);
    for (cudaStream_t x : r.side)
        if (x) cudaStreamSynchronize(x);
    if (r.stat) cudaStreamSynchronize(r.stat);
    cudaGetLastError();
}

gapsp_status fill_finish(FillRun& r, gapsp_stats* st) {
    gapsp_handle* h = r.h;
    cudaStream_t s = r.s;
    const size_t N = h->N;
    // (a fill that ran as a graph joined its side streams inside every
    // chunk; its events were recorded in the capture only)
    if (r.K > 0 && !r.graphed) {
        CK(cudaStreamWaitEvent(s, r.e_ahead[0], 0));
        CK(cudaStreamWaitEvent(s, r.e_ahead[1], 0));
    }
    if (r.stat && !r.graphed) {
        for (int k = 0; k < kDepRing; ++k) CK(cudaStreamWaitEvent(s, r.e_depth[k], 0));
    }
    CK(cudaEventRecord(h->ev1, s));
    unsigned long long hs[S_SLOTS];
    int sw = 0;
    CK(cudaMemcpyAsync(hs, h->stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&sw, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st) {
        st->propagations = hs[S_PROPAGATIONS];
        st->prepass_propagations = r.prepass;
        st->distance_ops = hs[S_OPS];
        st->new_pairs = hs[S_NEW] >> 1;
        st->rounds = hs[S_ROUNDS];
        st->prefilled_pairs = 0;
        st->sweeps = hs[S_SWEEPS];
        st->lines = hs[S_LINES];
        st->lookahead_propagations = hs[S_AHEAD];
        st->lookahead_hits = hs[S_HITS];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        st->ms_total = ms;
        if (st->round_new && st->round_new_cap) {
            const size_t n = std::min<uint64_t>(st->round_new_cap, hs[S_ROUNDS]);
            if (n) CK(cudaMemcpyAsync(st->round_new, h->round_new, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        }
        if (st->sources && st->sources_cap) {
            const size_t n = std::min<uint64_t>(st->sources_cap, hs[S_PROPAGATIONS]);
            if (n) CK(cudaMemcpyAsync(st->sources, h->sel_log, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        }
        if (h->kind == GAPSP_MASK) {
            // pairs in different components or touching an obstacle
            std::vector<int32_t> comp(N), size(N);
            CK(cudaMemcpyAsync(comp.data(), h->comp, N * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(size.data(), h->comp_size, N * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            uint64_t same = 0;
            for (size_t p = 0; p < N; ++p)
                if (comp[p] == (int32_t)p) same += (uint64_t)size[p] * (uint64_t)(size[p] - 1) / 2;
            st->prefilled_pairs = (uint64_t)N * (N - 1) / 2 - same;
        }
    }
    if (h->checked && sw == 0) {
        uint64_t bad = 0;
        const gapsp_status cs = certify_rows(h, r.Dd, nullptr, h->N, s, &bad);
        if (cs != GAPSP_OK) return cs;
        if (bad) {
            std::snprintf(t_detail, sizeof t_detail, "certificate: %llu entries of D break the distance equations",
                          (unsigned long long)bad);
            return GAPSP_E_CHECK;
        }
    }
    if (!r.d_dev) CK(cudaMemcpyAsync(r.D, r.Dd, N * N * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return status_from_word(sw);
}

bool valid_order(gapsp_order o) {
    return o == GAPSP_NAIVE || o == GAPSP_SPIRAL || o == GAPSP_MINFILL || o == GAPSP_EXTREMA ||
           o == GAPSP_REPULSION;
}

}  // namespace rt
}  // namespace gapsp

namespace gapsp {
namespace rt {

// The batched form as one CUDA graph. Each image's fill is set up on a
// worker stream of its own, then one chunk of its rounds (the round
// kernels, the lookahead branch, the depth-sum stream and the copies of its
// flags) is captured once into a graph; the chunks of all images are child
// graphs, side by side, of one graph, so that a single graph launch advances
// every image by one chunk. The host launches it one launch ahead of the
// one whose flags it reads, drops the images that are done (re-instantiating
// the graph without them) and stops when all are done. Rounds queued after
// an image is done find nothing to select and return at once, exactly as in
// gapsp_all_pairs, so every result and count equals that of the image alone.
struct BatchGraph {
    int n;
    std::vector<cudaStream_t> ws;
    std::vector<FillRun> runs;
    std::vector<cudaGraph_t> chunk;
    std::vector<uint64_t> per_chunk;  // kernel launches in one chunk of image i
    std::vector<int> replays;         // chunks image i has been launched with
    cudaStream_t ls = nullptr;        // the graph launches
    cudaGraphExec_t exec = nullptr;
    std::vector<int> in_exec;         // images of the instantiated graph
    cudaEvent_t ev[2] = {nullptr, nullptr};
    explicit BatchGraph(int n_) : n(n_), ws(n_, nullptr), runs(n_), chunk(n_, nullptr), per_chunk(n_, 0),
                                  replays(n_, 0) {}
    ~BatchGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaGraph_t g : chunk)
            if (g) cudaGraphDestroy(g);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (ls) cudaStreamDestroy(ls);
        for (cudaStream_t x : ws)
            if (x) cudaStreamDestroy(x);
    }
    // stream a waits for everything queued on stream b so far
    static cudaError_t order_after(cudaStream_t a, cudaStream_t b) {
        cudaEvent_t e = nullptr;
        cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r == cudaSuccess) r = cudaEventRecord(e, b);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(a, e, 0);
        if (e) cudaEventDestroy(e);
        return r;
    }
    gapsp_status instantiate(const std::vector<int>& imgs) {
        if (exec) {
            CK(cudaStreamSynchronize(ls));
            CK(cudaGraphExecDestroy(exec));
            exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaGraphCreate(&g, 0));
        for (int i : imgs) {
            cudaGraphNode_t node;
            const cudaError_t e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, chunk[i]);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                CK(e);
            }
        }
        const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        in_exec = imgs;
        return GAPSP_OK;
    }
    gapsp_status launch(int k) {
        CK(cudaGraphLaunch(exec, ls));
        CK(cudaEventRecord(ev[k & 1], ls));
        for (int i : in_exec) ++replays[i];
        return GAPSP_OK;
    }
    gapsp_status run(gapsp_handle* const* hs, gapsp_order order, uint32_t* const* Ds, gapsp_stats* st) {
        for (int i = 0; i < n; ++i) {
            CK(cudaStreamCreateWithFlags(&ws[i], cudaStreamNonBlocking));
            CK(order_after(ws[i], hs[i]->st));  // after the handle's own stream
            runs[i].h = hs[i];
            runs[i].order = order;
            runs[i].D = Ds[i];
            runs[i].s = ws[i];
            runs[i].sm_share = std::max(1, hs[i]->sms / n);  // the fills share the device
        }
        gapsp_status gs = GAPSP_OK;
        for (int i = 0; i < n && gs == GAPSP_OK; ++i) gs = fill_begin(runs[i]);
        for (int i = 0; i < n && gs == GAPSP_OK; ++i) {
            const uint64_t l0 = hs[i]->launches;
            runs[i].graphed = true;
            cudaError_t e = cudaStreamBeginCapture(ws[i], cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                gs = fill_enqueue(runs[i], kChunk, true);
                cudaGraph_t g = nullptr;
                e = cudaStreamEndCapture(ws[i], &g);
                chunk[i] = g;
                if (gs == GAPSP_OK && e != cudaSuccess) gs = GAPSP_E_CUDA;
            } else {
                gs = GAPSP_E_CUDA;
            }
            cudaGetLastError();
            per_chunk[i] = hs[i]->launches - l0;
            hs[i]->launches = l0;
        }
        if (gs == GAPSP_OK) {
            if (cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess)
                gs = GAPSP_E_CUDA;
            for (int i = 0; i < n && gs == GAPSP_OK; ++i)
                if (order_after(ls, ws[i]) != cudaSuccess) gs = GAPSP_E_CUDA;
        }
        std::vector<int> running;
        for (int i = 0; i < n; ++i) running.push_back(i);
        if (gs == GAPSP_OK) gs = instantiate(running);
        int launched = 0, waited = 0;
        if (gs == GAPSP_OK) gs = launch(launched++);
        while (gs == GAPSP_OK && !running.empty()) {
            if ((gs = launch(launched++)) != GAPSP_OK) break;
            // the flags of the launch before: every image of it has run
            // that chunk (a newer launch may have updated the flags since,
            // with values that only move towards "done")
            if (cudaEventSynchronize(ev[waited++ & 1]) != cudaSuccess) {
                gs = GAPSP_E_CUDA;
                break;
            }
            std::vector<int> still;
            for (int i : running) {
                gapsp_handle* h = hs[i];
                const gapsp_status dev = status_from_word(h->h_done[2]);
                if (dev != GAPSP_OK) gs = dev;
                else if (h->cancel.load()) gs = GAPSP_E_CANCELLED;
                else if (!h->h_done[0]) {
                    const int cap = h->max_rounds ? h->max_rounds : h->N + 2 + 64;
                    if ((waited)*kChunk >= cap) gs = GAPSP_E_TIMEOUT;
                    still.push_back(i);
                }
            }
            if (gs != GAPSP_OK) break;
            // re-instantiate without the images that are done once they
            // make up an eighth of the graph (their chunks cost launches)
            if (still.size() < running.size() && (running.size() - still.size()) * 8 >= in_exec.size()) {
                running = still;
                if (!running.empty()) gs = instantiate(running);
            } else {
                running = still;
            }
        }
        // every worker stream waits for the graph launches, then the fills
        // finish on them
        for (int i = 0; i < n; ++i) {
            if (!ws[i]) continue;
            if (ls && order_after(ws[i], ls) != cudaSuccess && gs == GAPSP_OK) gs = GAPSP_E_CUDA;
            hs[i]->launches += per_chunk[i] * (uint64_t)replays[i];
        }
        for (int i = 0; i < n && gs == GAPSP_OK; ++i) gs = fill_finish(runs[i], st ? st + i : nullptr);
        if (gs != GAPSP_OK) {
            if (ls) cudaStreamSynchronize(ls);
            for (int i = 0; i < n; ++i) fill_drain(runs[i]);
        }
        // the handles' streams are ordered after the batch
        for (int i = 0; i < n; ++i)
            if (ws[i]) order_after(hs[i]->st, ws[i]);
        cudaGetLastError();
        return gs;
    }
};

}  // namespace rt
}  // namespace gapsp

extern "C" {

gapsp_status gapsp_all_pairs(gapsp_handle* h, gapsp_order order, uint32_t* D, gapsp_stats* st) {
    if (!h || !D) return GAPSP_E_INVALID;
    if (!valid_order(order)) return GAPSP_E_INVALID;
    FillRun r;
    r.h = h;
    r.order = order;
    r.D = D;
    r.s = h->st;
    h->cancel.store(0);
    gapsp_status gs = fill_begin(r);
    if (gs == GAPSP_OK) gs = fill_enqueue(r, next_chunk(r));
    while (gs == GAPSP_OK && !r.finished) {
        if ((gs = fill_enqueue(r, next_chunk(r))) == GAPSP_OK) gs = fill_poll(r);
    }
    if (gs == GAPSP_OK) gs = fill_finish(r, st);
    if (gs != GAPSP_OK) fill_drain(r);
    return gs;
}

const char* gapsp_last_error_detail(void) { return t_detail; }

gapsp_status gapsp_certify(gapsp_handle* h, const uint32_t* D, const int32_t* sources, int K, uint64_t* bad) {
    if (!h || !D || !bad || K < 0 || (!sources && K > h->N)) return GAPSP_E_INVALID;
    *bad = 0;
    if (K == 0) return GAPSP_OK;
    if (!is_device_ptr(D)) return GAPSP_E_INVALID;
    int32_t* dsrc = nullptr;
    if (sources) {
        std::vector<int32_t> hs(K);
        CK(cudaMemcpyAsync(hs.data(), sources, (size_t)K * sizeof(int32_t), cudaMemcpyDefault, h->st));
        CK(cudaStreamSynchronize(h->st));
        for (int k = 0; k < K; ++k)
            if (hs[k] < 0 || hs[k] >= h->N) return GAPSP_E_INVALID;
        CK(dalloc(&dsrc, (size_t)K, h->st));
        const cudaError_t e = cudaMemcpyAsync(dsrc, hs.data(), (size_t)K * sizeof(int32_t), cudaMemcpyHostToDevice, h->st);
        if (e != cudaSuccess) {
            dfree(dsrc, h->st);
            CK(e);
        }
    }
    const gapsp_status gs = certify_rows(h, D, dsrc, K, h->st, bad);
    dfree(dsrc, h->st);
    return gs;
}

gapsp_status gapsp_cancel(gapsp_handle* h) {
    if (!h) return GAPSP_E_INVALID;
    h->cancel.store(1);
    return GAPSP_OK;
}

long long gapsp_debug_fail_alloc(int n) {
    g_fail_after.store(n < 0 ? -1 : n);
    return g_live.load();
}

gapsp_status gapsp_all_pairs_batch(gapsp_handle* const* hs, int n, gapsp_order order, uint32_t* const* Ds,
                                   gapsp_stats* st) {
    if (n < 0 || (n > 0 && (!hs || !Ds))) return GAPSP_E_INVALID;
    if (!valid_order(order)) return GAPSP_E_INVALID;
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !Ds[i]) return GAPSP_E_INVALID;
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return GAPSP_E_INVALID;  // one fill per handle
    }
    if (n == 0) return GAPSP_OK;
    for (int i = 0; i < n; ++i) hs[i]->cancel.store(0);
    BatchGraph bg(n);
    gapsp_status result = bg.run(hs, order, Ds, st);
    return result;
}

gapsp_status gapsp_profile_enable(gapsp_handle* h, int enable) {
    if (!h) return GAPSP_E_INVALID;
    h->prof = enable != 0;
    return GAPSP_OK;
}

gapsp_status gapsp_profile_trace(gapsp_handle* h, double* ms, uint64_t* launches, int32_t* kind,
                                 float* dur_ms, uint64_t cap, uint64_t* count) {
    if (!h || !ms || !launches) return GAPSP_E_INVALID;
    for (int k = 0; k < GAPSP_NUM_KERNELS; ++k) { ms[k] = 0.0; launches[k] = 0; }
    CK(cudaStreamSynchronize(h->st));
    uint64_t i = 0;
    for (auto& t : h->timed) {
        float e = 0.f;
        CK(cudaEventElapsedTime(&e, t.a, t.b));
        if (t.kind >= 0 && t.kind < GAPSP_NUM_KERNELS) { ms[t.kind] += e; launches[t.kind] += 1; }
        if (kind && dur_ms && i < cap) { kind[i] = t.kind; dur_ms[i] = e; }
        ++i;
        h->pool.push_back(t.a);
        h->pool.push_back(t.b);
    }
    if (count) *count = i;
    h->timed.clear();
    return GAPSP_OK;
}

gapsp_status gapsp_profile_read(gapsp_handle* h, double* ms, uint64_t* launches) {
    return gapsp_profile_trace(h, ms, launches, nullptr, nullptr, 0, nullptr);
}

}  // extern "C"
