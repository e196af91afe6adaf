// gapsp_tune: picks the launch parameters of an image's fill by measuring
// them (declared in include/gapsp.h).
//
// The candidates are the parameters that shape the work on the GPU without
// changing D: sources per round B in {16, ..., 1024} (how many trees a round
// builds and fills: wider rounds make the chain of rounds shorter and cost
// more propagations),
// whether rows are computed ahead (the lookahead launches), and the tree
// fill variant: walks one lane at a time with marks in global memory (0) or
// in lockstep (-1), rows of marks staged in shared memory (8, for B <= 32),
// and for B >= 128 the first round written one-sided and mirrored (-2, -3),
// which only pays when that round fills most pairs. Each candidate fills the
// caller's image once after a warm-up fill, timed with events on a stream of
// its own; the fastest wins.
// Results are kept in a text cache, one line per key (H, W, conn, kind,
// order, multiprocessor count), so that each shape is measured once.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gapsp.h"
#include "internal.h"
#include "runtime.h"

using namespace gapsp;
using namespace gapsp::rt;

namespace {

std::mutex g_tune_mu;  // one tuning (and cache update) at a time per process

struct Key {
    int H, W, conn, kind, order, sms;
    bool operator==(const Key& o) const {
        return H == o.H && W == o.W && conn == o.conn && kind == o.kind && order == o.order && sms == o.sms;
    }
};

struct Choice {
    int B, lookahead, fill_rows;
    double ms;
};

bool cache_lookup(const char* path, const Key& k, Choice& c) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        Key x{};
        Choice y{};
        if (std::sscanf(line, "gapsp-tune-2 %d %d %d %d %d %d %d %d %d %lf", &x.H, &x.W, &x.conn, &x.kind, &x.order,
                        &x.sms, &y.B, &y.lookahead, &y.fill_rows, &y.ms) == 10 &&
            x == k) {
            c = y;  // the last line for a key wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, const Key& k, const Choice& c) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "gapsp-tune-2 %d %d %d %d %d %d %d %d %d %.4f\n", k.H, k.W, k.conn, k.kind, k.order, k.sms, c.B,
                 c.lookahead, c.fill_rows, c.ms);
    std::fclose(f);
}

// Device time of one fill with these options (after a warm-up fill on the
// same handle), or a negative value if the fill failed.
double time_fill(const uint8_t* img, const uint8_t* mask, int H, int W, gapsp_opts o, gapsp_order order,
                 uint32_t* D, cudaStream_t st) {
    o.stream = st;
    gapsp_handle* h = nullptr;
    if (gapsp_create(img, H, W, mask, &o, &h) != GAPSP_OK) return -1.0;
    double ms = -1.0;
    gapsp_stats s{};
    if (gapsp_all_pairs(h, order, D, &s) == GAPSP_OK && gapsp_all_pairs(h, order, D, &s) == GAPSP_OK)
        ms = s.ms_total;
    gapsp_destroy(h);
    return ms;
}

}  // namespace

extern "C" gapsp_status gapsp_tune(const uint8_t* img, const uint8_t* mask, int H, int W, const gapsp_opts* base,
                                   gapsp_order order, const char* cache_path, gapsp_opts* best, double* best_ms) {
    if (!best || !valid_order(order)) return GAPSP_E_INVALID;
    if (H < 1 || W < 1 || H > GAPSP_MAX_SIDE || W > GAPSP_MAX_SIDE || H * W > GAPSP_MAX_N) return GAPSP_E_INVALID;
    gapsp_opts o;
    gapsp_default_opts(&o);
    if (base) o = *base;
    if (o.conn == 0) o.conn = 8;
    if (o.kind == GAPSP_MASK ? !mask : !img) return GAPSP_E_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    const Key key{H, W, o.conn, (int)o.kind, (int)order, sms};
    std::lock_guard<std::mutex> lock(g_tune_mu);
    Choice c{};
    if (!cache_lookup(cache_path, key, c)) {
        // measure every candidate on a scratch array of the image's size
        const size_t N = (size_t)H * W;
        cudaStream_t st = nullptr;
        uint32_t* D = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return GAPSP_E_CUDA;
        }
        if (dalloc(&D, N * N, st) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamDestroy(st);
            return GAPSP_E_NOMEM;
        }
        const int Bs[] = {16, 32, 64, 128, 256, 512, 1024};
        const int looks[] = {0, -1};
        const int fills[] = {0, -1, 8, -2, -3};
        c.ms = -1.0;
        for (int B : Bs)
            for (int la : looks)
                for (int fr : fills) {
                    // staged rows only pay with few trees per round, the
                    // one-sided first round only with many; from B = 256 on,
                    // no multiprocessor is left for lookahead launches
                    if ((fr == 8 && B > 32) || (fr <= -2 && B < 128) || (la == -1 && B >= 256)) continue;
                    gapsp_opts t = o;
                    t.B = B;
                    t.lookahead = la;
                    t.fill_rows = fr;
                    const double ms = time_fill(img, mask, H, W, t, order, D, st);
                    if (ms >= 0 && (c.ms < 0 || ms < c.ms)) c = Choice{B, la, fr, ms};
                }
        dfree(D, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (c.ms < 0) return GAPSP_E_CUDA;
        cache_store(cache_path, key, c);
    }
    *best = o;
    best->B = c.B;
    best->lookahead = c.lookahead;
    best->fill_rows = c.fill_rows;
    best->stream = base ? base->stream : nullptr;
    if (best_ms) *best_ms = c.ms;
    return GAPSP_OK;
}
