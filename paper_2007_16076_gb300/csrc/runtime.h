// Internal runtime of gapsp, shared by the C ABI (gapsp.cu) and the
// request server (server.cu): the handle, the allocation helpers, and one
// all-pairs fill in progress with the steps that advance it. Not part of
// the public C ABI.
#pragma once
#include <chrono>
#include <atomic>
#include <vector>

#include "internal.h"

struct gapsp_handle {
    int H = 0, W = 0, N = 0, conn = 8, kind = 0, B = 32;
    uint64_t seed = 0;
    size_t budget = 0;
    cudaStream_t st = nullptr;
    int tiles_w = 0, tiles_h = 0, words = 0;
    int sweep_phases = 0;
    int fill_rows = 0;
    int prop_blocks = 0;
    int lookahead = 0;  // option: 0 auto, -1 off, else candidates per round
    bool warm = true;   // option: propagations start from complete neighbour rows
    bool checked = false;  // option: certify every result (certify.cu)
    unsigned long long* bad = nullptr;  // certificate's violation count
    int max_sweep_rounds = 0;  // option: 0 = N + 2
    int max_rounds = 0;        // option: 0 = N + 66
    std::atomic<int> cancel{0};  // gapsp_cancel: stop the all-pairs call in progress
    int sms = 0;        // multiprocessors of the device
    uint64_t launches = 0;
    // image
    uint8_t* f = nullptr;
    uint32_t* pgeo = nullptr;
    int32_t* tbase = nullptr;
    uint8_t* bound = nullptr;
    int32_t* comp = nullptr;
    int32_t* comp_size = nullptr;
    int* status = nullptr;
    int* changed = nullptr;
    // fill state
    bool fill_ready = false;
    uint32_t* cnt = nullptr;
    uint32_t* cnt_base = nullptr;
    unsigned long long* marks = nullptr;
    int32_t* parent = nullptr;
    ulonglong2* seg = nullptr;
    int32_t* jmp = nullptr;
    int32_t* acc = nullptr;
    int32_t* sel = nullptr;
    int* nsel = nullptr;
    int* cursor = nullptr;
    int* done = nullptr;
    int32_t* seq = nullptr;
    int32_t* rank = nullptr;
    int32_t* grank = nullptr;
    uint8_t* row_done = nullptr;  // [N]: row already written by a propagation
    uint8_t* row_claim = nullptr; // [N]: row handed to a lookahead launch (done or in flight)
    int32_t* rp_ring = nullptr;   // spiral with repulsion: turns, S, draw state
    int32_t* rp_fstart = nullptr;
    uint8_t* rp_fcyc = nullptr;
    unsigned* rp_inS = nullptr;
    gapsp::RepState* rp_state = nullptr;
    uint8_t* rp_taken = nullptr;
    int32_t* cand = nullptr;      // [2][1024]: lookahead candidates, by round parity
    int* ncand = nullptr;         // [2]
    uint16_t* dep_exit = nullptr; // [ring][B][N] (N <= 16384): trees handed to k_depths, by round
    uint16_t* dep_size = nullptr; // [ring][B][N]
    int* dep_count = nullptr;     // [ring]
    unsigned long long* stats = nullptr;
    unsigned long long* round_new = nullptr;
    unsigned long long* last_new = nullptr;
    uint32_t* vfloor = nullptr;   // selection: least leading key field at the previous round
    int32_t* sel_log = nullptr;
    uint32_t* emap = nullptr;
    uint32_t* gmap = nullptr;
    unsigned long long* best = nullptr;
    uint8_t* cen = nullptr;
    int* h_done = nullptr;  // pinned, [4]: "done" flag, then the status word, after an even /
                            // odd chunk of rounds
    // scratch for host-side arrays
    uint32_t* Dtmp = nullptr;
    size_t Dtmp_bytes = 0;
    int32_t* src_dev = nullptr;
    int src_cap = 0;
    uint32_t* out_tmp = nullptr;
    size_t out_tmp_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // per-kernel timing (gapsp_profile_*)
    bool prof = false;
    struct Timed { int kind; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> pool;
};

namespace gapsp {
namespace rt {

// Depth-sum hand-over buffers per handle: a ring of this many rounds (a
// chunk of rounds is a whole number of turns of the ring).
constexpr int kDepRing = 4;

// Host-side fault injection and the count of live allocations
// (gapsp_debug_fail_alloc).
extern std::atomic<long long> g_live;
bool injected_failure();

// Device memory comes from the stream-ordered allocator: allocated on the
// stream whose work uses it first, freed on the handle's stream after the
// work queued there. Neither call waits for the device, so creating and
// destroying handles does not stall other handles' work in flight (plain
// cudaFree synchronises the whole device).
template <class T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 1, st);
    if (e == cudaSuccess) g_live.fetch_add(1);
    else *p = nullptr;
    return e;
}

template <class T>
void dfree(T*& p, cudaStream_t st) {
    if (p) {
        cudaFreeAsync(p, st);
        g_live.fetch_sub(1);
    }
    p = nullptr;
}

// Pinned host words (four per call) from a process-wide pool.
cudaError_t halloc(int** p);
void hfree(int*& p);

// Certificate of K rows of D on stream st (row k = d(src[k], .), src a
// device array or NULL for rows 0..K-1): *bad receives the count of
// entries that break the distance equations.
gapsp_status certify_rows(gapsp_handle* h, const uint32_t* D, const int32_t* src, int K, cudaStream_t st,
                          uint64_t* bad);

// Propagation arguments common to every launch on this handle.
PropArgs base_prop(const gapsp_handle* h);
// Device bytes of the fill state of a handle (marks, trees, counts).
size_t fill_state_bytes(const gapsp_handle* h);

// One fill in progress: the state of gapsp_all_pairs between its steps, so
// that several fills (one per image) can advance side by side.
// Host clock in seconds (steady).
inline double host_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct FillRun {
    gapsp_handle* h = nullptr;
    gapsp_order order = GAPSP_MINFILL;
    uint32_t* D = nullptr;   // caller's array
    uint32_t* Dd = nullptr;  // device array the kernels fill
    bool d_dev = true;
    cudaStream_t s = nullptr;
    int nseq = 0;
    uint64_t prepass = 0;
    SelectArgs sa{};
    RepArgs ra{};
    PropArgs pa{};
    TreeArgs ta{};
    int rounds = 0;
    bool finished = false;
    bool graphed = false;  // its chunks run as a captured graph (gapsp_all_pairs_batch)
    int sm_share = 0;      // multiprocessors the fill plans its lookahead for (0: all)
    bool one_side_first = false;  // the first round writes one side of its pairs, then mirrors them
    // lookahead: the next K candidates of each round are propagated on a
    // second stream while the round's tree and fill run
    int K = 0;
    PropArgs pa_ahead{};
    cudaStream_t side[2] = {nullptr, nullptr};  // lookahead launches of even / odd rounds
    cudaEvent_t e_sel = nullptr;
    cudaEvent_t e_ahead[2] = {nullptr, nullptr};  // lookahead launch of an even / odd round
    // chunks of rounds: the host keeps one chunk queued beyond the one whose
    // "done" flag it waits for, so that the device never waits for the host
    cudaEvent_t chunk_ev[2] = {nullptr, nullptr};
    int chunks = 0, polled = 0;
    int chunk_rounds[2] = {0, 0};  // rounds of the chunks in flight, by parity
    double t_poll = 0.0;           // host clock (s) at the previous poll (or the fill's start)
    double round_s = 0.0;          // host time per round of the last chunk polled
    // depth sums (N <= 16384) on a third, low-priority stream: a round's
    // trees are handed over in a buffer of the round's parity, which the
    // tree launch two rounds later waits for
    cudaStream_t stat = nullptr;
    cudaEvent_t e_tree[kDepRing] = {}, e_depth[kDepRing] = {};
    FillRun() = default;
    FillRun(const FillRun&) = delete;
    FillRun& operator=(const FillRun&) = delete;
    ~FillRun() {
        if (e_sel) cudaEventDestroy(e_sel);
        for (cudaEvent_t e : e_ahead)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : chunk_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : e_tree)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : e_depth)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t x : side)
            if (x) cudaStreamDestroy(x);
        if (stat) cudaStreamDestroy(stat);
    }
};

// Rounds per chunk: small enough that the rounds queued after the fill is
// done cost little, large enough that the host stays ahead of the device.
constexpr int kChunk = 8;
static_assert(kChunk % kDepRing == 0, "a chunk of rounds is a whole number of turns of the depth ring");
// Rounds of the next chunk of a fill that is not captured in a graph: 1, 1,
// 2, 4, then kChunk, so that a fill done in its first rounds (a round with
// many sources can fill every pair) queues few rounds past its end; and at
// most 2 once rounds take over half a millisecond (two such rounds keep the
// device busy while the host polls, and fewer rounds run past the end).
inline int next_chunk(const FillRun& r) {
    const int grow = r.chunks < 2 ? 1 : r.chunks < 4 ? 1 << (r.chunks - 1) : kChunk;
    return r.round_s > 0.5e-3 && grow > 2 ? 2 : grow;
}

// Set-up of a fill: checks D, allocates what is missing, initialises the
// state on r.s, runs the extrema pre-pass of the ranked orders.
gapsp_status fill_begin(FillRun& r);
// Enqueues `chunk` rounds and an asynchronous copy of the "done" flag and
// the status word. With `graph`, the rounds are being captured into a graph
// that is launched again and again: the chunk then joins its side streams at
// its end and writes its flags to the first slots, and no chunk event is
// recorded.
gapsp_status fill_enqueue(FillRun& r, int chunk, bool graph = false);
// Whether the oldest chunk not yet polled has completed (fill_poll would
// return without waiting).
bool fill_chunk_ready(const FillRun& r);
// Waits for the oldest chunk not yet polled, reads its flags; sets
// r.finished; returns a device error, the round limit or a cancellation.
gapsp_status fill_poll(FillRun& r);
// After the last chunk: joins the side streams, reads the counts into st,
// copies a host D back; synchronous.
gapsp_status fill_finish(FillRun& r, gapsp_stats* st);
// After an error: waits for everything the fill queued.
void fill_drain(FillRun& r);
bool valid_order(gapsp_order o);

}  // namespace rt
}  // namespace gapsp
