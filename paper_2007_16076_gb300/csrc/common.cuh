// Device-side definitions shared by the gapsp kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gapsp {

// Sentinel for "not reached yet" inside the sweeps. Real distances are below
// (GAPSP_MAX_N - 1) * 511 < 2^26, and the sentinel plus any edge weight or
// line prefix stays below 2^31, so all sweep arithmetic is plain int32.
constexpr int PINF = 0x3FFFFFFF;
constexpr uint32_t UNREACH = 0xFFFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;

// Bits of the device status word.
constexpr int ST_NOT_CONVERGED = 1;
constexpr int ST_BAD_SOURCE = 2;
constexpr int ST_TIMEOUT = 4;

// Device counters of a fill run (one uint64 each).
enum StatSlot {
    S_PROPAGATIONS = 0,
    S_OPS = 1,
    S_NEW = 2,     // twice the new pairs: each filled pair adds one mark to each of its rows
    S_ROUNDS = 3,
    S_SWEEPS = 4,  // total sweeps run by the propagation warps
    S_LINES = 5,   // lines processed (not skipped) by the propagation warps
    S_AHEAD = 6,   // lookahead propagations run (rows computed ahead of their round)
    S_HITS = 7,    // selected sources whose row had been computed ahead
    S_SLOTS = 8
};

// Marks: one 64-bit word per (row, 8x8 pixel tile), stored tile-major (the
// words of one tile for all rows, then the next tile), so that the words of
// neighbouring rows for the same tile are adjacent. Bit (r%8)*8 + (c%8) of
// row b's word for tile (r/8)*tiles_w + c/8 says whether the pair
// {b, (r,c)} is filled.

// Programmatic dependent launch: a kernel launched after another on the
// same stream with the programmatic-serialization attribute may start while
// its predecessor drains; it waits here before touching the predecessor's
// results (a no-op for a kernel launched without the attribute). The trigger
// lets the successor's blocks be scheduled once every block of this kernel
// has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ int ld_cg(const int* p) {
    int v;
    asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned long long ld_cg64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

}  // namespace gapsp
