// Internal interfaces between the host runtime and the kernel translation
// units of gapsp. Not part of the public C ABI.
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gapsp.h"
#include "common.cuh"

namespace gapsp {

// Whether p is device (or managed) memory that kernels may address.
bool is_device_ptr(const void* p);

// Status of a call from the device status word (ST_* bits).
inline gapsp_status status_from_word(int w) {
    if (w & ST_NOT_CONVERGED) return GAPSP_E_NOT_CONVERGED;
    if (w & ST_TIMEOUT) return GAPSP_E_TIMEOUT;
    if (w & ST_BAD_SOURCE) return GAPSP_E_INVALID;
    return GAPSP_OK;
}

// Runs set() once per device, the device current at the call: kernel
// attributes such as the dynamic shared-memory limit belong to a device, so
// a process that uses several GPUs sets them on each. `done` holds one bit
// per device (devices beyond 63 set them on every call). Two threads may
// both run set() the first time; the attribute calls are idempotent.
template <class F>
inline void once_per_device(std::atomic<unsigned long long>& done, F&& set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 64;
    }
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return;
    set();
    if (bit) done.fetch_or(bit, std::memory_order_release);
}

struct PropArgs {
    int* map_base;              // distance maps (int32 view of uint32 rows)
    const int32_t* map_row;     // job j writes map_base + map_row[j] * N (NULL: j * N)
    const int32_t* sources;     // job j's single source (NULL: seed_flags)
    const uint8_t* seed_flags;  // multi-source seeds, one job (NULL: single sources)
    const int* njobs_dev;       // device-side job count (NULL: use njobs)
    int njobs;
    int H, W, N, conn, kind_mask;
    int level_bytes;            // bytes per level: 1, or 2 for the channel sum (GAPSP_SUM)
    const uint8_t* f;           // levels (uint8, or uint16 for GAPSP_SUM) or free flags (mask)
    int* status;                // device status word (ST_* bits)
    unsigned long long* sweeps; // optional: total sweeps run
    int max_sweeps;
    int convert;                // write UNREACH for pixels never reached
    int phases;                 // warps per sweep direction (1, 2 or 4)
    int cluster;                // blocks (row strips) per source: 1, 2 or 4
    uint8_t* row_done;          // [N] or NULL: skip sources whose row is already in the
                                // output; set the flag once a row is written
    unsigned long long* ran;    // or NULL: counts the jobs that were not skipped
    unsigned long long* hits;   // or NULL: counts the jobs skipped by row_done
    // Warm start (fills only; NULL: the map starts from the seeds alone): the
    // distances array, row q at warm_rows + q * N, holding at every entry
    // either an upper bound of the distance (a path's cost, mostly the exact
    // distance) or UNREACH. The map of source s starts from row s and from
    // d(s,q) + d(q,x) for its neighbours q.
    const uint32_t* warm_rows;
};

// Picks the per-lane width and launches kernel (a).
cudaError_t launch_propagate(const PropArgs& a, int conn, int kind, int grid, int warps_per_block,
                             cudaStream_t st);
// Values held per lane for lines of length up to `side`.
int prop_vpl(int side);
// Blocks (one cluster) a single-source propagation of this image uses.
int prop_blocks_per_job(const PropArgs& a);
// Whether the distance map of a propagation lives in shared memory (else it
// is the output row itself, in global memory).
bool prop_map_in_smem(const PropArgs& a);

struct ImagePrep {
    const uint8_t* f;
    int H, W, conn, kind;
    uint8_t* bound;  // boundary flags: free pixels with fewer free neighbours than conn
    uint32_t* pgeo;  // [N]: tile << 8 | bit of each pixel (from k_geometry)
    int32_t* tbase;  // [tiles]: pixel index of each tile's top-left pixel
    int tiles_w, tiles;
};
cudaError_t launch_image_prep(const ImagePrep& p, cudaStream_t st);

struct TreeArgs {
    int H, W, N, conn, kind, tiles_w, words;
    unsigned wdiv;              // ceil(2^32 / W) (0 when W = 1): row of p = umulhi(p, wdiv)
    const uint8_t* f;
    const uint32_t* D;          // the array; row sel[j] holds d(sel[j], .)
    const int32_t* sel;         // selected sources
    const int* nsel;            // device count
    const uint32_t* pgeo;       // [N]: tile << 8 | bit of each pixel
    const int32_t* tbase;       // [words]: top-left pixel of each tile
    int32_t* parent;            // [B][N] (N > 16384 only)
    ulonglong2* seg;            // [B][N]: x = mask of the tile segment; y = exit vertex + 1
                                // (0 past the root, bits 0-16) | its tile (bits 17-26), and
                                // the same for the next segment's exit (bits 27-53)
    int32_t* jmp;               // [2][B][N] scratch for the depth pointer jumping
    int32_t* acc;               // [2][B][N] scratch for the depth pointer jumping
    unsigned long long* marks;  // [words][N]: tile t's word of row b at t * N + b
    uint32_t* cnt;              // [N]
    const uint32_t* cnt_base;   // [N] fill count at the start (1 + pairs no path joins)
    uint32_t* Dw;               // writable array for new pairs
    unsigned long long* stats;  // StatSlot counters
    int rows_per_block;         // 0: marks in global memory; -1: walks in lockstep; else staged rows
    int one_side;               // lockstep only: write D[a][b] (a the ancestor) and not D[b][a]
    // N <= 16384: the depth sums are left to k_depths; the tree hands it the
    // segment exits (+1) and segment sizes of each tree, and the tree count
    uint16_t* dep_exit;         // [B][N] or NULL (then the tree sums depths itself)
    uint16_t* dep_size;         // [B][N]
    int* dep_count;
};
// pdl: launched as a programmatic dependent of the previous kernel on st
cudaError_t launch_tree(const TreeArgs& a, int B, cudaStream_t st, bool pdl = false);
// Distance operations of the trees handed over by a tree launch (N <= 16384).
cudaError_t launch_depths(const TreeArgs& a, int B, cudaStream_t st);
cudaError_t launch_fill(const TreeArgs& a, int B, cudaStream_t st, bool pdl = false);
// Shared memory of a fill block: its rows of marks (padded by one word) and
// one "changed" byte per word (rows padded by four bytes).
__host__ __device__ inline int fill_row_stride(int words) { return words + 1; }
__host__ __device__ inline int fill_chg_stride(int words) { return words + 4; }
__host__ __device__ inline size_t fill_smem_bytes(int rows, int words) {
    return (size_t)rows * (fill_row_stride(words) * 8 + fill_chg_stride(words));
}
cudaError_t launch_recount(const TreeArgs& a, cudaStream_t st, bool pdl = false);
// Completes the pairs a one-sided fill left: D[i][j] = D[j][i] where only one is known.
cudaError_t launch_mirror(uint32_t* D, int N, cudaStream_t st);

struct SelectArgs {
    int N, B, order;            // 0 naive / 1 spiral (sequence), 2 minfill, 3 extrema
    const uint32_t* cnt;
    const int32_t* rank;        // minfill: position in Ext
    const int32_t* grank;       // extrema: free points strictly farther from the centroid
    const int32_t* seq;         // naive / spiral sequence
    int nseq;
    int* cursor;                // sequence cursor
    int32_t* sel;
    int* nsel;
    unsigned long long* stats;
    unsigned long long* round_new_log;  // per-round new pairs (reads S_NEW)
    unsigned long long* last_new;       // S_NEW value at the previous round
    int32_t* sel_log;           // sources in selection order (capacity N)
    int* done;                  // set to 1 once every point is filled
    int32_t* cand;              // lookahead candidates (capacity K), or NULL
    int* ncand;                 // device count of candidates, or NULL
    int K;                      // candidates wanted: rows not computed yet
    int KL;                     // ranking positions after the selection they are taken
                                // from (B + KL <= 1024)
    const uint8_t* row_done;    // [N]: rows already computed
    uint8_t* row_claim;         // [N]: rows handed to a lookahead launch; set for each candidate
    uint32_t* vfloor;           // minfill / extrema (N <= 16384): the least leading key field (cnt,
                                // or grank) among the unfilled points at the previous selection;
                                // 0 at the start. It never decreases.
};
cudaError_t launch_select(const SelectArgs& a, cudaStream_t st);

// Spiral with repulsion: the turns (rings of free pixels, clockwise), the
// current turn's list S as a bit per ring position, and the draw state.
struct RepState {
    unsigned long long rng;     // SplitMix64 state
    int cur;                    // current turn, -1 = none
    int nframes;
};
struct RepArgs {
    const int32_t* ring;        // [N] pixels of all turns, turn after turn
    const int32_t* fstart;      // [nframes + 1]
    const uint8_t* fcyc;        // [nframes]: closed ring (else an open line)
    unsigned* inS;              // [32]: bit i of word i/32 = ring position i of the current turn in S
    RepState* state;
    uint8_t* taken;             // [N]: drawn in the current round
};
cudaError_t launch_select_repulsion(const SelectArgs& a, const RepArgs& r, cudaStream_t st);

struct InitArgs {
    int N;
    uint32_t* D;
    uint32_t* cnt;
    const int32_t* comp;        // component label per pixel (-1 obstacle), or NULL
    const int32_t* comp_size;   // per label
    int full_init;              // write UNREACH everywhere first (mask variant)
};
cudaError_t launch_init(const InitArgs& a, cudaStream_t st);

struct ExtremaArgs {
    int N;
    const uint8_t* freef;       // NULL: every pixel free
    const int32_t* comp;        // NULL: one component
    const uint32_t* e;          // distance from the boundary
    unsigned long long* best;   // [N] per component label: packed (e, -p)
    uint8_t* cen_flags;         // [N] centroid seeds
    const uint32_t* g;          // distance from the centroids
    int32_t* rank;              // [N]
    int32_t* grank;             // [N]
    unsigned long long* keys;   // N > 16384: sort scratch, N rounded up to 16384 keys, or NULL
};
cudaError_t launch_centroids(const ExtremaArgs& a, cudaStream_t st);
cudaError_t launch_rank(const ExtremaArgs& a, cudaStream_t st);

struct CompArgs {
    int H, W, conn;
    const uint8_t* freef;
    int32_t* label;
    int32_t* size;
    int* changed;
    int* status;
};
cudaError_t launch_components(const CompArgs& a, cudaStream_t st);

cudaError_t launch_unreach_convert(uint32_t* rows, size_t n, cudaStream_t st);

// The certificate of a result (certify.cu): row k of D (rows x N, row-major)
// holds d(src[k], .) (src NULL: k); bad counts the entries that break
// d(p,p) = 0, d(p,r) = min over neighbours q of d(p,q) + w(q,r).
struct CertifyArgs {
    const uint32_t* D;
    int rows;
    const int32_t* src;
    int H, W, N, conn, kind;
    const uint8_t* f;           // levels (16-bit for kind 3) or free flags
    unsigned long long* bad;
};
cudaError_t launch_certify(const CertifyArgs& a, cudaStream_t st);
// F(p) = sum over the L channels (planes of N bytes) of the levels of p.
cudaError_t launch_channel_sum(const uint8_t* planes, int L, int N, uint16_t* F, cudaStream_t st);

}  // namespace gapsp
