/*
 * gapsp: all pairs of geodesic distances on a grey image, on one GB300 GPU.
 *
 * The operation is the one of Noyel, Angulo & Jeulin, "Fast computation of
 * all pairs of geodesic distances":
 *   - pixels are the vertices of a graph whose edges join 4- or 8-neighbours
 *     (Sec. 2, eqs. "voisinage 1/2");
 *   - an edge between neighbours p and q costs w(p,q) = f(p) + f(q) + 1, the
 *     sum-of-grey-levels pseudo-metric of Sec. 2 (eq. "distance somme") plus
 *     one so that every edge costs at least 1. Diagonal steps cost the same
 *     as axial ones (a 3x3 neighbourhood, no Euclidean correction, Sec. 3);
 *   - the distance d(p,q) is the minimum over paths of the summed edge costs
 *     (Sec. 2, eqs. "temps" and "distance");
 *   - the N x N array D is filled by geodesic propagations from chosen source
 *     points plus Property 1 (Sec. 2): along the geodesic tree of a
 *     propagation from s, d(a,b) = d(s,b) - d(s,a) for every ancestor a of b;
 *   - sources are chosen in naive (raster) order, spiral order (Sec. 3.1,
 *     Algorithm "spiral method"), spiral order with repulsion (Sec. 3.2: a
 *     source drawn on the current turn takes its two neighbours on each side
 *     of the turn out of the draw), by decreasing distance from the geodesic
 *     centroid with ties to the least filled point (Sec. 3.3, Algorithm
 *     "geodesic extrema method") or by minimum filling rate with ties to the
 *     greatest geodesic extremum (Sec. 3.4, Algorithm "method based on the
 *     filling rate"); the last two take the extrema pre-pass of Sec. 3.3 (two
 *     more propagations).
 *
 * Two more edge costs are included: the L1 pseudo-metric of Sec. 2 (eq.
 * "distance abs difference"), w = |f(p) - f(q)| + 1, and an obstacle mask:
 * w = 2 between free pixels, obstacle pixels have no edges, and pairs that no
 * path joins hold GAPSP_UNREACH.
 *
 * Data layout. Images are H x W, row-major, pixel p = r*W + c, N = H*W.
 * D is row-major uint32 N x N: D[p*N + q] = d(p,q). D[p][p] = 0, D is
 * symmetric, unreachable pairs hold GAPSP_UNREACH. D does not depend on the
 * order or on B: only the counts in gapsp_stats do.
 *
 * Errors. Every call returns a status and never aborts, traps or hangs:
 * device loops carry iteration limits and report GAPSP_E_NOT_CONVERGED /
 * GAPSP_E_TIMEOUT through a status word instead.
 *
 * Threading. A handle is used by one host thread at a time. Calls are
 * ordered on opts.stream (NULL = the legacy default stream) and return when
 * their results are complete.
 */
#ifndef GAPSP_H
#define GAPSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GAPSP_UNREACH 0xFFFFFFFFu

/* Largest supported image side, and largest N = H*W. */
#define GAPSP_MAX_SIDE 256
#define GAPSP_MAX_N 65536

typedef struct gapsp_handle gapsp_handle; /* opaque */

typedef enum {
    GAPSP_OK = 0,
    GAPSP_E_INVALID = 1,        /* bad argument: sizes, pointers, sources, order */
    GAPSP_E_NOMEM = 2,          /* a device or host allocation failed */
    GAPSP_E_BUDGET = 3,         /* the call's footprint exceeds opts.mem_budget */
    GAPSP_E_CUDA = 4,           /* a CUDA runtime call failed */
    GAPSP_E_NOT_CONVERGED = 5,  /* a propagation hit its sweep limit */
    GAPSP_E_TIMEOUT = 6,        /* a round loop hit its round limit */
    GAPSP_E_CANCELLED = 7,      /* gapsp_cancel stopped the call */
    GAPSP_E_CHECK = 8           /* the result failed its certificate (opts.checked) */
} gapsp_status;

typedef enum {
    GAPSP_NAIVE = 0,   /* raster order, filled points skipped (Sec. 1 with the tree) */
    GAPSP_SPIRAL = 1,  /* Sec. 3.1, Algorithm "spiral method" */
    GAPSP_MINFILL = 2, /* Sec. 3.4, Algorithm "method based on the filling rate" */
    GAPSP_EXTREMA = 3, /* Sec. 3.3, Algorithm "geodesic extrema method" */
    GAPSP_REPULSION = 4 /* Sec. 3.2, Algorithm "spiral method with repulsion", h = 3 */
} gapsp_order;

typedef enum {
    GAPSP_GREY = 0, /* w(p,q) = f(p) + f(q) + 1: sum of grey levels (Sec. 2, eq. "distance somme") */
    GAPSP_MASK = 1, /* w = 2 between free pixels; obstacles have no edges */
    GAPSP_L1 = 2,   /* w(p,q) = |f(p) - f(q)| + 1: pseudo-metric L1 (Sec. 2, eq. "distance abs difference") */
    GAPSP_SUM = 3   /* multichannel image of L channels (Sec. 2: values in T^L): the sum pseudo-metric
                       over the channels, w(p,q) = sum_l (f_l(p) + f_l(q)) + 1 = F(p) + F(q) + 1 with
                       F = sum_l f_l; handles of this kind come from gapsp_create_channels */
} gapsp_kind;

typedef struct {
    int conn;          /* 4 or 8 (0 = 8) */
    gapsp_kind kind;   /* GAPSP_GREY, GAPSP_MASK or GAPSP_L1 (GAPSP_SUM: gapsp_create_channels) */
    int B;             /* sources per round, 1..1024 (0 = 32) */
    uint64_t seed;     /* seed of the spiral orders' draws */
    size_t mem_budget; /* bytes of device memory a call may use (0 = no limit) */
    int sweep_phases;  /* warps per sweep direction in a propagation: 0 = auto, 1, 2 or 4 */
    int fill_rows;     /* tree fill variant (D is the same for all):
                          0 = marks claimed in global memory (the default);
                          1..32 = rows of marks staged in shared memory per block;
                          -1 = every round walks in lockstep, one warp per half
                               tile and tree;
                          -2 = as 0, but the first round walks in lockstep and
                               writes one side of each pair, and one pass over D
                               mirrors it (pays when the first round fills most
                               pairs: many sources per round, B >= 128);
                          -3 = as -1, with the first round as in -2 */
    int checked;       /* 1: certify every result before returning it (gapsp_certify on the
                          whole D or on the rows; about one more read of the array);
                          a result that fails returns GAPSP_E_CHECK. 0: off */
    void *stream;      /* cudaStream_t the calls run on (NULL = default stream) */
    int prop_blocks;   /* blocks (row strips, one thread-block cluster) per propagation:
                          0 = auto, 1, 2 or 4 */
    int lookahead;     /* gapsp_all_pairs: candidates per round whose rows are
                          computed ahead, on a second stream, while the round's
                          trees fill D: 0 = auto (one per multiprocessor the round's
                          B sources leave free), -1 = none, else 1..1024-B. The
                          candidates are the next points in the order's ranking
                          at the round's start; a later round whose source was
                          computed ahead skips that propagation. D and every count
                          are the same with or without it. */
    int warm_start;    /* gapsp_all_pairs: 0 = on, -1 = off. A propagation starts from
                          the complete rows of its source's filled neighbours q
                          (d(s,x) <= d(q,s) + d(q,x)) instead of from the source
                          alone; exact once every neighbour is filled. D and every
                          count are the same either way. */
    int max_sweep_rounds; /* iteration limit of one propagation: rounds in which every
                          line is swept once in each of the four directions; 0 = N + 2,
                          which no propagation needs to reach (a shortest path has at
                          most N - 1 turns). Reaching it ends the propagation and the
                          call returns GAPSP_E_NOT_CONVERGED. */
    int max_rounds;    /* gapsp_all_pairs: limit on the rounds of the loop; 0 = N + 66,
                          above what any order needs (every round fills at least its
                          first source's row). Reaching it ends the call with
                          GAPSP_E_TIMEOUT. Both limits are checked between chunks of
                          8 rounds. */
} gapsp_opts;

typedef struct {
    uint64_t propagations;         /* sources propagated by the round loop */
    uint64_t prepass_propagations; /* +2 for the extrema pre-pass (Sec. 3.3-3.4) */
    uint64_t distance_ops;         /* sum over propagations of the depth of every reached vertex */
    uint64_t new_pairs;            /* pairs filled by the tree fills */
    uint64_t rounds;               /* rounds of the loop */
    uint64_t prefilled_pairs;      /* pairs no path joins (mask variant), filled at init */
    double ms_total;               /* device time of the call */
    uint64_t *round_new;           /* optional, caller-owned host array: new pairs per
                                      round (capacity round_new_cap), or NULL */
    uint64_t round_new_cap;
    int32_t *sources;              /* optional, caller-owned host array receiving the
                                      sources in selection order (capacity sources_cap) */
    uint64_t sources_cap;
    uint64_t sweeps;               /* directional sweeps run by all propagations */
    uint64_t lines;                /* image lines those sweeps processed (the rest were
                                      skipped as unchanged) */
    uint64_t lookahead_propagations; /* rows computed ahead of their round (opts.lookahead);
                                        not part of `propagations` */
    uint64_t lookahead_hits;       /* propagations whose row had been computed ahead */
} gapsp_stats;

/* Fills *opts with the defaults (conn 8, grey, B 32, seed 0, no budget). */
void gapsp_default_opts(gapsp_opts *opts);

/*
 * Creates a handle for one image (Sec. 2: the image as a graph).
 *   img  : H*W uint8 grey levels, row-major, host or device pointer; read
 *          during the call only (copied).
 *   mask : H*W uint8, 1 = free pixel, 0 = obstacle; host or device; required
 *          for GAPSP_MASK and ignored for GAPSP_GREY and GAPSP_L1.
 *   H, W : 1..GAPSP_MAX_SIDE each, H*W <= GAPSP_MAX_N.
 * The handle owns a device copy of the image, its tile geometry and the
 * bookkeeping arrays (marks, fill counts). On error *out is
 * NULL and nothing is allocated.
 */
gapsp_status gapsp_create(const uint8_t *img, int H, int W, const uint8_t *mask,
                          const gapsp_opts *opts, gapsp_handle **out);

/*
 * Creates a handle for a multichannel image with the sum pseudo-metric over
 * its channels (GAPSP_SUM; Sec. 2 extends the pseudo-metrics to images with
 * values in T^L): w(p,q) = sum_l (f_l(p) + f_l(q)) + 1.
 *   planes : L*H*W uint8, channel after channel, each H*W row-major; host or
 *            device pointer, read during the call only.
 *   L      : 1..GAPSP_MAX_CHANNELS; with N = H*W, (N - 1) * (510 * L + 1) must
 *            stay below 2^30 - 2^18 (every distance fits the kernels' int32
 *            sweeps; always true up to 32 channels).
 * opts.kind is ignored (GAPSP_SUM). The handle then serves gapsp_all_pairs,
 * gapsp_all_pairs_batch and gapsp_rows like any other. Errors as gapsp_create.
 */
#define GAPSP_MAX_CHANNELS 32
gapsp_status gapsp_create_channels(const uint8_t *planes, int L, int H, int W, const gapsp_opts *opts,
                                   gapsp_handle **out);

/*
 * Fills the whole N x N array D (Sec. 2, eq. "A": all (N^2 - N)/2 pairs) by
 * propagations from sources chosen in `order`, B per round, plus the
 * geodesic-tree fill of Property 1.
 *   D  : caller-owned uint32 N*N, device pointer or host pointer (a host
 *        array is filled through a device buffer the call allocates). A
 *        device D must be 16-byte aligned (rows move 16 bytes at a time).
 *   st : may be NULL; otherwise receives the counts, which equal those of
 *        the same order simulated on the CPU.
 * Errors: GAPSP_E_INVALID (order, NULL or misaligned D), GAPSP_E_BUDGET, GAPSP_E_NOMEM,
 * GAPSP_E_NOT_CONVERGED, GAPSP_E_TIMEOUT, GAPSP_E_CUDA. On error the content
 * of D is unspecified.
 */
gapsp_status gapsp_all_pairs(gapsp_handle *h, gapsp_order order, uint32_t *D,
                             gapsp_stats *st);

/*
 * Batched form: fills the arrays of n images at once, one handle and one
 * caller-owned array D[i] per image (device or host pointers, as for
 * gapsp_all_pairs), all in the same order. The round loops of the images run
 * side by side on one worker stream per image, so many small images keep
 * the GPU busy together; every result and count equals that of
 * gapsp_all_pairs on the image alone. The work is ordered after each
 * handle's stream and each handle's stream is ordered after it.
 *   st : NULL or n entries.
 * Errors: GAPSP_E_INVALID (n < 0, NULL pointers, a handle given twice), and
 * those of gapsp_all_pairs; on error the arrays are unspecified.
 */
gapsp_status gapsp_all_pairs_batch(gapsp_handle *const *h, int n, gapsp_order order,
                                   uint32_t *const *D, gapsp_stats *st);

/*
 * Single-source propagations (Sec. 1: "geodesic propagation"): out[k*N + q]
 * = d(sources[k], q) for k < K. No tree, marks or selection.
 *   sources : K int32 pixel indices, host or device pointer.
 *   out     : caller-owned uint32 K*N, device or host pointer; a device
 *             out must be 16-byte aligned.
 * Errors: GAPSP_E_INVALID (K < 0, a source outside [0, N), NULL pointers, a
 * misaligned device out),
 * GAPSP_E_BUDGET, GAPSP_E_NOMEM, GAPSP_E_NOT_CONVERGED, GAPSP_E_CUDA. With
 * an invalid source nothing is written.
 */
gapsp_status gapsp_rows(gapsp_handle *h, const int32_t *sources, int K, uint32_t *out);

/*
 * Certificate of a result, independent of how it was computed. With positive
 * integer edge weights the distances from p are the unique solution of
 * d(p,p) = 0 and d(p,r) = min over the neighbours q of r of d(p,q) + w(q,r)
 * for r != p (Sec. 2, eqs. "temps" and "distance": a shortest path ends
 * with an edge), UNREACH when no neighbour is reachable. The call checks
 * every entry of the K rows given against that equation, on the device, and
 * so proves the rows exact when it counts no violation.
 *   D       : K*N uint32, device pointer, row k = d(sources[k], .).
 *   sources : K int32 host or device, or NULL for rows 0..K-1 (the whole
 *             array when K = N).
 *   bad     : receives the number of entries that break the equation.
 * Returns GAPSP_OK (whatever *bad is), GAPSP_E_INVALID, GAPSP_E_CUDA.
 */
gapsp_status gapsp_certify(gapsp_handle *h, const uint32_t *D, const int32_t *sources, int K,
                           uint64_t *bad);

/* Releases the handle and its device memory. NULL is accepted. The memory
 * is released in stream order, after the work queued on the handle's
 * stream, without waiting for it; a handle that staged a host array (a
 * host D or host rows) first waits for its stream. */
void gapsp_destroy(gapsp_handle *h);

/*
 * Asks the gapsp_all_pairs or gapsp_all_pairs_batch call running on h in
 * another host thread to stop. The request is seen between chunks of 8
 * rounds: the call then waits for the work it has queued and returns
 * GAPSP_E_CANCELLED, and D is unspecified. Each all-pairs call clears the
 * request when it starts, so a cancel with no call running has no effect.
 * Safe to call from any thread while the handle is alive.
 */
gapsp_status gapsp_cancel(gapsp_handle *h);

/* Static text for a status code. */
const char *gapsp_strerror(gapsp_status s);

/* The CUDA runtime call behind this host thread's last GAPSP_E_CUDA or
 * GAPSP_E_NOMEM from a handle call: source line, the call and the runtime's
 * error text ("" if none). Valid until this thread's next failing call. */
const char *gapsp_last_error_detail(void);

/* Number of kernels the library launched on this handle since its creation
 * (for launch accounting). */
uint64_t gapsp_kernel_launches(const gapsp_handle *h);

/*
 * Per-kernel device time, for measurement. While enabled, every launch of
 * the kernels below is bracketed by CUDA events on the handle's stream, and
 * gapsp_profile_read returns, per kernel, the summed event time (ms) and the
 * number of launches since the last read (then resets). Enabling adds two
 * event records per launch; leave it off for throughput timing.
 * Kernel ids: 0 selection (c), 1 propagation (a), 2 tree: parents,
 * segments and depths (a'), 3 lookahead propagations (on the second stream,
 * overlapping the others), 4 tree fill (b), 5 init, 6 extrema pre-pass
 * helpers, 7 depth sums of the trees (N <= 16384, on a third stream), 8
 * fill-count update, 9 completion of a one-sided first round (the mirror
 * pass).
 * ms and launches: caller-owned arrays of GAPSP_NUM_KERNELS entries.
 */
#define GAPSP_NUM_KERNELS 10
gapsp_status gapsp_profile_enable(gapsp_handle *h, int enable);
gapsp_status gapsp_profile_read(gapsp_handle *h, double *ms, uint64_t *launches);
/* Like gapsp_profile_read, and also returns the individual launches in
 * launch order: kind[i] (kernel id) and dur_ms[i], for i < min(cap, count);
 * *count receives the number of launches recorded. */
gapsp_status gapsp_profile_trace(gapsp_handle *h, double *ms, uint64_t *launches,
                                 int32_t *kind, float *dur_ms, uint64_t cap, uint64_t *count);

/*
 * Rows without any allocation. The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they call
 * (an engine that owns the device through its own fixed pool, code where an
 * allocation would stall the device or a latency budget, a host whose
 * allocator is not the CUDA runtime's). It computes the same rows as
 * gapsp_rows, needs no handle and allocates nothing: its only scratch (the
 * device copy of the source list and a status word) is one fixed array of
 * GAPSP_NOALLOC_MAX_SOURCES * 4 + 256 bytes that every GPU loading the
 * library holds until the process exits.
 *   img     : H*W uint8, DEVICE pointer: grey levels (GAPSP_GREY, GAPSP_L1) or free
 *             flags, nonzero = free (GAPSP_MASK).
 *   sources : K int32 pixel indices, host or device pointer.
 *   out     : caller-owned DEVICE uint32 K*N, 16-byte aligned; out[k*N + q] =
 *             d(sources[k], q).
 *   stream  : cudaStream_t the work runs on (NULL = default stream); the call
 *             waits for it and returns when the rows are complete.
 * Limits: 0 <= K <= GAPSP_NOALLOC_MAX_SOURCES; H, W and N as gapsp_create.
 * Errors: GAPSP_E_INVALID for sizes beyond the limits, a NULL pointer, an
 * img or out that is not device memory, a misaligned out or a source outside
 * [0, N) (nothing is written then); GAPSP_E_NOT_CONVERGED; GAPSP_E_CUDA.
 * Every call shares the one array and it keeps the last call's contents:
 * calls that overlap on the GPU race, so order them on one stream. The first
 * call on a device looks up the array's address on that device; make it
 * before any stream capture.
 */
#define GAPSP_NOALLOC_MAX_SOURCES 4096
gapsp_status gapsp_rows_noalloc(const uint8_t *img, int H, int W, int conn, gapsp_kind kind,
                                const int32_t *sources, int K, uint32_t *out, void *stream);

/*
 * Autotuner for the launch parameters of one image's fill. The paper has no
 * counterpart: its method is the same for every choice, and D is too; only
 * the time and the counts of B > 1 change. Measures, on the image given, a
 * fill in `order` for every candidate of B in {16, 32, ..., 1024}, lookahead on
 * (0) or off (-1; only below B = 256, where the rounds leave multiprocessors
 * free) and the tree fill variants (fill_rows 0 and -1; 8 for B <= 32; -2
 * and -3 for B >= 128), and returns in *best the options
 * of *base (NULL: the defaults) with the fastest candidate's B, lookahead
 * and fill_rows; *best_ms (may be NULL) receives its device time.
 *   img, mask : as gapsp_create (host or device).
 *   cache_path: NULL, or a text file of earlier results keyed by (H, W,
 *               conn, kind, order, multiprocessor count): a key found there
 *               is not measured again; a new result is appended.
 * Allocates a scratch N x N array while measuring. Errors: GAPSP_E_INVALID,
 * GAPSP_E_NOMEM, GAPSP_E_CUDA (no candidate could run).
 */
gapsp_status gapsp_tune(const uint8_t *img, const uint8_t *mask, int H, int W, const gapsp_opts *base,
                        gapsp_order order, const char *cache_path, gapsp_opts *best, double *best_ms);

/*
 * Serving: a request loop with continuous batching. The paper has no
 * serving layer; this runs its operations (Sec. 1: rows d(s, .); Sec. 2-3:
 * the all-pairs fill in any order) for many callers at once.
 *
 * gapsp_server_submit queues a request (its inputs are copied, so the
 * caller's arrays may be freed at once) and returns its id. A scheduler
 * thread inside the library admits queued requests in arrival order as soon
 * as one of opts.slots slots (one CUDA stream each) is free and the
 * request's footprint fits in what the memory budget leaves: the footprint
 * is its result, N*N*4 bytes for an all-pairs fill or K*N*4 bytes for K
 * rows, plus the working state it holds while it runs (the image state, and
 * the marks, trees and counts of a fill). Admitted requests run side by side
 * on the GPU: a fill advances chunk by chunk of rounds and requests that
 * arrive while others run start as soon as a slot and memory free up. A
 * request whose footprint exceeds the whole budget is rejected at once
 * (GAPSP_E_BUDGET). Each result equals that of gapsp_all_pairs / gapsp_rows
 * on the same image alone (D does not depend on the order; the counts are
 * the order's).
 *
 * Results stay resident in device memory, counted against the budget, until
 * gapsp_server_release. A request with out == NULL gets a result array the
 * server allocates (gapsp_result.result) and frees at release; with a
 * caller-owned device out, the caller keeps that array alive until the
 * request is done. The server uses the CUDA device current at its creation.
 * All calls may come from any host thread.
 */
typedef struct gapsp_server gapsp_server;

typedef enum { GAPSP_REQ_ALL_PAIRS = 0, GAPSP_REQ_ROWS = 1 } gapsp_request_kind;

typedef struct {
    gapsp_request_kind kind;
    const uint8_t *img;     /* H*W host array: grey levels (GAPSP_GREY, GAPSP_L1) */
    const uint8_t *mask;    /* H*W host array: 1 = free (GAPSP_MASK), else NULL */
    int H, W, conn;         /* as gapsp_create */
    gapsp_kind img_kind;
    gapsp_order order;      /* GAPSP_REQ_ALL_PAIRS */
    const int32_t *sources; /* GAPSP_REQ_ROWS: K host pixel indices in [0, N) */
    int K;                  /* GAPSP_REQ_ROWS: 1 .. GAPSP_MAX_N */
    uint32_t *out;          /* NULL, or a caller-owned 16-byte aligned device array of
                               N*N (all-pairs) or K*N (rows) uint32 */
} gapsp_request;

typedef struct {
    size_t mem_budget;  /* device bytes the admitted requests may hold at once (0 = 120 GiB) */
    int slots;          /* requests running at once, one stream each: 1..256 (0 = 16) */
    int B;              /* sources per round of the fills (0 = 256: fewer rounds, lower latency) */
    int lookahead;      /* as gapsp_opts.lookahead, for the fills */
} gapsp_server_opts;

typedef struct {
    uint64_t id;
    int done;                  /* 1 once the request has finished (status is final) */
    gapsp_status status;
    uint32_t *result;          /* device array holding the result (valid until release) */
    size_t result_bytes;
    size_t footprint;          /* bytes the request was admitted with */
    double t_submit_ms, t_admit_ms, t_done_ms; /* server clock, from its creation */
    uint64_t propagations;     /* the fill's propagations (rows: K) */
    uint64_t rounds;
} gapsp_result;

typedef struct {
    uint64_t submitted, rejected, admitted, completed, failed, queued;
    size_t bytes_in_use, peak_bytes, budget;
} gapsp_server_counts;

void gapsp_server_default_opts(gapsp_server_opts *opts);
/* Starts a server (and its scheduler thread) on the current device. */
gapsp_status gapsp_server_create(const gapsp_server_opts *opts, gapsp_server **out);
/* Queues a request. Errors: GAPSP_E_INVALID (sizes, kinds, pointers, a source
 * outside [0, N)), GAPSP_E_BUDGET (footprint above the whole budget). */
gapsp_status gapsp_server_submit(gapsp_server *s, const gapsp_request *req, uint64_t *id);
/* Waits up to timeout_ms (< 0: no limit) for request id to finish; fills *out.
 * GAPSP_E_TIMEOUT if it has not finished in time, GAPSP_E_INVALID for an id
 * unknown or released. */
gapsp_status gapsp_server_wait(gapsp_server *s, uint64_t id, int timeout_ms, gapsp_result *out);
/* Up to cap requests finished since the last poll, each reported once;
 * returns how many. */
int gapsp_server_poll(gapsp_server *s, gapsp_result *out, int cap);
/* Copies a finished request's result (result_bytes) into dst, host or
 * device memory; returns when the copy is complete. */
gapsp_status gapsp_server_read(gapsp_server *s, uint64_t id, void *dst, size_t bytes);
/* Frees a finished request's result and its share of the budget. */
gapsp_status gapsp_server_release(gapsp_server *s, uint64_t id);
gapsp_status gapsp_server_stats(gapsp_server *s, gapsp_server_counts *c);
/* Stops the server: requests running finish, requests still queued are
 * cancelled (GAPSP_E_CANCELLED), and every result not yet released is freed.
 * Results held by the client count against the budget: a client that waits
 * for a request while holding the results whose memory it needs waits
 * forever, so release results as they complete (gapsp_server_poll). */
void gapsp_server_destroy(gapsp_server *s);

/*
 * Host-side fault injection, for tests of the error paths: after n more
 * successful device or pinned-host allocations made by the library, the
 * next one fails as if the device were out of memory (the call returns
 * GAPSP_E_NOMEM and frees what it had allocated). n < 0 turns it off (the
 * default). Process-wide; nothing on the GPU is made to fail. Returns the
 * number of device and pinned-host allocations the library holds (all
 * handles together), so that a test can see that a failed call leaked
 * nothing.
 */
long long gapsp_debug_fail_alloc(int n);

#ifdef __cplusplus
}
#endif

#endif /* GAPSP_H */
