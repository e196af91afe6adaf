// gapsp_server: a request loop that serves all-pairs fills and row queries
// on one GPU with continuous batching (declared in include/gapsp.h).
//
// Requests are submitted from any host thread and queued in arrival order.
// A scheduler thread admits the request at the head of the queue as soon as
// one of the server's slots (one CUDA stream each) is free and its footprint
// (result + working state) fits in what the memory budget leaves; admitted
// requests run side by side, each on its own slot stream:
//   - a row query is one propagation launch of its K sources (Sec. 1),
//     finished when an event recorded after it has completed;
//   - an all-pairs fill (Sec. 2-3) advances chunk by chunk: whenever the
//     oldest queued chunk of rounds of a fill has completed, the scheduler
//     reads its flags and queues the next one, so fills admitted at
//     different times interleave their rounds on the GPU, and a request that
//     arrives while others run starts as soon as a slot frees.
// Nothing here waits for the whole device: handles and results come from
// the stream-ordered allocator. A result stays resident in device memory,
// counted against the budget, until the client releases it.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gapsp.h"
#include "internal.h"
#include "runtime.h"

using namespace gapsp;
using namespace gapsp::rt;

namespace {

struct Request {
    uint64_t id = 0;
    gapsp_request req{};             // sizes and kinds; pointers below are the server's copies
    std::vector<uint8_t> img, mask;
    std::vector<int32_t> src;
    size_t out_bytes = 0, work_bytes = 0;
    bool own_out = true;
    double t_submit = 0, t_admit = 0, t_done = -1;
    gapsp_status status = GAPSP_OK;
    int slot = -1;
    gapsp_handle* h = nullptr;
    uint32_t* out = nullptr;
    int32_t* dsrc = nullptr;
    std::unique_ptr<FillRun> run;
    cudaEvent_t ev = nullptr;
    int* hstat = nullptr;
    gapsp_stats st{};
};

double now_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Device bytes a request holds while it runs, besides its result: the
// handle's image state, and the fill state of an all-pairs request.
size_t working_bytes(const gapsp_request& q, int B) {
    const size_t N = (size_t)q.H * q.W;
    const size_t words = (size_t)((q.H + 7) / 8) * ((q.W + 7) / 8);
    size_t b = N * 32 + 4096;
    if (q.kind == GAPSP_REQ_ROWS) return b + (size_t)q.K * 4;
    b += N * words * 8 + (size_t)B * N * (4 + 16 + 8 + 8) + N * 96 + 2 * 1024 * 4 + 4096;
    if (N <= 16384) b += 8 * (size_t)B * N;
    return b;
}

}  // namespace

struct gapsp_server {
    gapsp_server_opts o{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> live;  // submitted and not yet released
    std::deque<uint64_t> completed;               // completed and not yet polled
    std::vector<cudaStream_t> streams;
    std::vector<char> busy;
    size_t used = 0, peak = 0;
    uint64_t next_id = 1, n_submitted = 0, n_rejected = 0, n_admitted = 0, n_completed = 0, n_failed = 0;
    bool stop = false;
    std::thread worker;

    void run_loop();
    void begin(Request* r);
    bool advance(Request* r);
    void finish(Request* r, gapsp_status s);
};

namespace {

void fill_result(const Request* r, gapsp_result* out) {
    std::memset(out, 0, sizeof(*out));
    out->id = r->id;
    out->done = r->t_done >= 0;
    out->status = r->status;
    out->result = r->out;
    out->result_bytes = r->out_bytes;
    out->footprint = r->out_bytes + r->work_bytes;
    out->t_submit_ms = r->t_submit;
    out->t_admit_ms = r->t_admit;
    out->t_done_ms = r->t_done;
    out->propagations = r->st.propagations;
    out->rounds = r->st.rounds;
}

}  // namespace

void gapsp_server::begin(Request* r) {
    cudaStream_t s = streams[r->slot];
    const gapsp_request& q = r->req;
    gapsp_opts go;
    gapsp_default_opts(&go);
    go.conn = q.conn;
    go.kind = q.img_kind;
    go.B = o.B;
    go.lookahead = o.lookahead;
    go.stream = s;
    gapsp_status gs = gapsp_create(q.img_kind == GAPSP_MASK ? nullptr : r->img.data(), q.H, q.W,
                                   q.img_kind == GAPSP_MASK ? r->mask.data() : nullptr, &go, &r->h);
    if (gs != GAPSP_OK) return finish(r, gs);
    const size_t N = (size_t)q.H * q.W;
    if (!r->out) {
        if (dalloc(&r->out, r->out_bytes / 4, s) != cudaSuccess) return finish(r, GAPSP_E_NOMEM);
        r->own_out = true;
    }
    if (q.kind == GAPSP_REQ_ROWS) {
        if (dalloc(&r->dsrc, (size_t)q.K, s) != cudaSuccess) return finish(r, GAPSP_E_NOMEM);
        if (halloc(&r->hstat) != cudaSuccess) return finish(r, GAPSP_E_NOMEM);
        if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) return finish(r, GAPSP_E_CUDA);
        PropArgs a = base_prop(r->h);
        a.map_base = (int*)r->out;
        a.sources = r->dsrc;
        a.njobs = q.K;
        a.convert = q.img_kind == GAPSP_MASK;
        a.phases = q.K > 304 ? 1 : 4;
        if (cudaMemcpyAsync(r->dsrc, r->src.data(), (size_t)q.K * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(r->h->status, 0, sizeof(int), s) != cudaSuccess ||
            launch_propagate(a, q.conn, q.img_kind, q.K, 1, s) != cudaSuccess ||
            cudaMemcpyAsync(r->hstat, r->h->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaEventRecord(r->ev, s) != cudaSuccess) {
            cudaGetLastError();
            return finish(r, GAPSP_E_CUDA);
        }
        r->h->launches += 1;
        r->st.propagations = (uint64_t)q.K;
        return;
    }
    (void)N;
    r->run.reset(new FillRun());
    FillRun& f = *r->run;
    f.h = r->h;
    f.order = q.order;
    f.D = r->out;
    f.s = s;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        f.sm_share = std::max(1, sms / (int)busy.size());  // the slots share the device
    cudaGetLastError();
    if ((gs = fill_begin(f)) == GAPSP_OK && (gs = fill_enqueue(f, next_chunk(f))) == GAPSP_OK)
        gs = fill_enqueue(f, next_chunk(f));
    if (gs != GAPSP_OK) {
        fill_drain(f);
        return finish(r, gs);
    }
}

// One step of a running request without waiting; true if it moved.
bool gapsp_server::advance(Request* r) {
    if (r->req.kind == GAPSP_REQ_ROWS) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) return false;
        if (q != cudaSuccess) {
            cudaGetLastError();
            finish(r, GAPSP_E_CUDA);
        } else {
            finish(r, status_from_word(*r->hstat));
        }
        return true;
    }
    FillRun& f = *r->run;
    if (!fill_chunk_ready(f)) return false;
    gapsp_status gs = fill_poll(f);
    if (gs == GAPSP_OK && f.finished) {
        gs = fill_finish(f, &r->st);
        if (gs != GAPSP_OK) fill_drain(f);
        finish(r, gs);
        return true;
    }
    if (gs == GAPSP_OK) gs = fill_enqueue(f, next_chunk(f));
    if (gs != GAPSP_OK) {
        fill_drain(f);
        finish(r, gs);
    }
    return true;
}

// Ends a request: frees its working state (stream-ordered), keeps the
// result (or frees it on error), and reports it.
void gapsp_server::finish(Request* r, gapsp_status s) {
    cudaStream_t st = streams[r->slot];
    r->run.reset();
    if (r->h) gapsp_destroy(r->h);
    r->h = nullptr;
    dfree(r->dsrc, st);
    hfree(r->hstat);
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    r->status = s;
    used -= r->work_bytes;
    if (s != GAPSP_OK) {
        if (r->own_out) dfree(r->out, st);
        r->out = nullptr;
        used -= r->out_bytes;
        r->out_bytes = 0;
        ++n_failed;
    }
    r->t_done = now_ms(t0);
    busy[r->slot] = 0;
    completed.push_back(r->id);
    ++n_completed;
    cv_done.notify_all();
    cv_work.notify_one();
}

void gapsp_server::run_loop() {
    cudaSetDevice(device);
    std::vector<Request*> active;
    for (;;) {
        std::vector<Request*> starting;
        {
            std::unique_lock<std::mutex> lock(mu);
            for (;;) {
                // admission: the head of the queue, when a slot is free and
                // its footprint fits in what the budget leaves
                while (!pending.empty()) {
                    Request* r = pending.front();
                    int slot = -1;
                    for (int i = 0; i < (int)busy.size(); ++i)
                        if (!busy[i]) { slot = i; break; }
                    if (slot < 0 || used + r->out_bytes + r->work_bytes > o.mem_budget) break;
                    pending.pop_front();
                    busy[slot] = 1;
                    r->slot = slot;
                    used += r->out_bytes + r->work_bytes;
                    if (used > peak) peak = used;
                    r->t_admit = now_ms(t0);
                    ++n_admitted;
                    starting.push_back(r);
                }
                if (!starting.empty() || !active.empty()) break;
                if (stop) {
                    // requests still queued when the server stops are
                    // cancelled (their memory may be held by results the
                    // client has not released)
                    while (!pending.empty()) {
                        Request* r = pending.front();
                        pending.pop_front();
                        r->status = GAPSP_E_CANCELLED;
                        r->out = nullptr;
                        r->out_bytes = 0;
                        r->t_done = now_ms(t0);
                        completed.push_back(r->id);
                        ++n_completed;
                        ++n_failed;
                    }
                    cv_done.notify_all();
                    return;
                }
                cv_work.wait(lock);
            }
        }
        for (Request* r : starting) {
            active.push_back(r);
            begin(r);
        }
        bool moved = false;
        for (size_t i = 0; i < active.size();) {
            Request* r = active[i];
            if (r->t_done < 0) moved |= advance(r);
            if (r->t_done >= 0) {
                active[i] = active.back();
                active.pop_back();
                moved = true;
            } else {
                ++i;
            }
        }
        if (!moved) {
            // nothing completed: wait a little, or until a request arrives
            std::unique_lock<std::mutex> lock(mu);
            if (pending.empty() || active.size() == busy.size())
                cv_work.wait_for(lock, std::chrono::microseconds(30));
        }
    }
}

extern "C" {

void gapsp_server_default_opts(gapsp_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mem_budget = (size_t)120 << 30;
    o->slots = 16;
    o->B = 256;  // wide rounds: a fill in fewer, shorter rounds (measured best for latency)
}

gapsp_status gapsp_server_create(const gapsp_server_opts* opts, gapsp_server** out) {
    if (!out) return GAPSP_E_INVALID;
    *out = nullptr;
    gapsp_server_opts o;
    gapsp_server_default_opts(&o);
    if (opts) o = *opts;
    if (o.mem_budget == 0) o.mem_budget = (size_t)120 << 30;
    if (o.slots == 0) o.slots = 16;
    if (o.B == 0) o.B = 256;
    if (o.slots < 1 || o.slots > 256 || o.B < 1 || o.B > 1024 || o.lookahead < -1 || o.lookahead > 1024)
        return GAPSP_E_INVALID;
    gapsp_server* s = new (std::nothrow) gapsp_server();
    if (!s) return GAPSP_E_NOMEM;
    s->o = o;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return GAPSP_E_CUDA;
    }
    s->streams.assign(o.slots, nullptr);
    s->busy.assign(o.slots, 0);
    for (int i = 0; i < o.slots; ++i)
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : s->streams)
                if (x) cudaStreamDestroy(x);
            delete s;
            return GAPSP_E_CUDA;
        }
    s->worker = std::thread([s] { s->run_loop(); });
    *out = s;
    return GAPSP_OK;
}

gapsp_status gapsp_server_submit(gapsp_server* s, const gapsp_request* q, uint64_t* id) {
    if (!s || !q || !id) return GAPSP_E_INVALID;
    *id = 0;
    if (q->H < 1 || q->W < 1 || q->H > GAPSP_MAX_SIDE || q->W > GAPSP_MAX_SIDE || q->H * q->W > GAPSP_MAX_N)
        return GAPSP_E_INVALID;
    if (q->conn != 4 && q->conn != 8) return GAPSP_E_INVALID;
    if (q->img_kind != GAPSP_GREY && q->img_kind != GAPSP_MASK && q->img_kind != GAPSP_L1) return GAPSP_E_INVALID;
    if (q->kind != GAPSP_REQ_ALL_PAIRS && q->kind != GAPSP_REQ_ROWS) return GAPSP_E_INVALID;
    if (q->img_kind == GAPSP_MASK ? !q->mask : !q->img) return GAPSP_E_INVALID;
    if (q->out && (reinterpret_cast<uintptr_t>(q->out) & 15)) return GAPSP_E_INVALID;
    const int N = q->H * q->W;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return GAPSP_E_NOMEM;
    r->req = *q;
    if (q->kind == GAPSP_REQ_ROWS) {
        if (q->K < 1 || !q->sources) return GAPSP_E_INVALID;
        r->src.assign(q->sources, q->sources + q->K);
        for (int32_t v : r->src)
            if (v < 0 || v >= N) return GAPSP_E_INVALID;
        r->out_bytes = (size_t)q->K * N * 4;
    } else {
        if (!valid_order(q->order)) return GAPSP_E_INVALID;
        r->out_bytes = (size_t)N * N * 4;
    }
    if (q->img_kind == GAPSP_MASK) r->mask.assign(q->mask, q->mask + N);
    else r->img.assign(q->img, q->img + N);
    r->work_bytes = working_bytes(*q, s->o.B);
    r->out = q->out;
    r->own_out = q->out == nullptr;
    r->req.img = nullptr;
    r->req.mask = nullptr;
    r->req.sources = nullptr;
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->n_submitted;
    if (s->stop) return GAPSP_E_INVALID;
    if (r->out_bytes + r->work_bytes > s->o.mem_budget) {
        ++s->n_rejected;
        return GAPSP_E_BUDGET;
    }
    r->id = s->next_id++;
    r->t_submit = now_ms(s->t0);
    *id = r->id;
    s->live[r->id] = r.get();
    s->pending.push_back(r.release());
    s->cv_work.notify_one();
    return GAPSP_OK;
}

gapsp_status gapsp_server_wait(gapsp_server* s, uint64_t id, int timeout_ms, gapsp_result* out) {
    if (!s || !out) return GAPSP_E_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end()) return GAPSP_E_INVALID;
    Request* r = it->second;
    auto done = [r] { return r->t_done >= 0; };
    if (timeout_ms < 0) s->cv_done.wait(lock, done);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done)) {
        fill_result(r, out);
        return GAPSP_E_TIMEOUT;
    }
    fill_result(r, out);
    return GAPSP_OK;
}

int gapsp_server_poll(gapsp_server* s, gapsp_result* out, int cap) {
    if (!s || !out || cap <= 0) return 0;
    std::lock_guard<std::mutex> lock(s->mu);
    int n = 0;
    while (n < cap && !s->completed.empty()) {
        auto it = s->live.find(s->completed.front());
        s->completed.pop_front();
        if (it == s->live.end()) continue;  // released already
        fill_result(it->second, out + n);
        ++n;
    }
    return n;
}

gapsp_status gapsp_server_read(gapsp_server* s, uint64_t id, void* dst, size_t bytes) {
    if (!s || !dst) return GAPSP_E_INVALID;
    uint32_t* src = nullptr;
    cudaStream_t st = nullptr;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->live.find(id);
        if (it == s->live.end() || it->second->t_done < 0 || it->second->status != GAPSP_OK) return GAPSP_E_INVALID;
        if (bytes != it->second->out_bytes) return GAPSP_E_INVALID;
        src = it->second->out;
        st = s->streams[it->second->slot];
    }
    // the result is complete (the request is done); the copy goes on the
    // request's slot stream and the call waits for it
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    return GAPSP_OK;
}

gapsp_status gapsp_server_release(gapsp_server* s, uint64_t id) {
    if (!s) return GAPSP_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end() || it->second->t_done < 0) return GAPSP_E_INVALID;
    Request* r = it->second;
    if (r->own_out && r->out) dfree(r->out, s->streams[r->slot]);
    s->used -= r->out_bytes;
    s->live.erase(it);
    delete r;
    s->cv_work.notify_one();
    return GAPSP_OK;
}

gapsp_status gapsp_server_stats(gapsp_server* s, gapsp_server_counts* c) {
    if (!s || !c) return GAPSP_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    c->submitted = s->n_submitted;
    c->rejected = s->n_rejected;
    c->admitted = s->n_admitted;
    c->completed = s->n_completed;
    c->failed = s->n_failed;
    c->queued = s->pending.size();
    c->bytes_in_use = s->used;
    c->peak_bytes = s->peak;
    c->budget = s->o.mem_budget;
    return GAPSP_OK;
}

void gapsp_server_destroy(gapsp_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();  // the requests queued or running complete first
    for (auto& kv : s->live) {
        Request* r = kv.second;
        if (r->own_out && r->out) dfree(r->out, s->streams[r->slot >= 0 ? r->slot : 0]);
        delete r;
    }
    s->live.clear();
    for (cudaStream_t x : s->streams) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
    }
    delete s;
}

}  // extern "C"
