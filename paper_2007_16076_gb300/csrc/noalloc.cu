// gapsp_rows_noalloc: single-source propagations that allocate nothing.
//
// Some callers cannot allocate device memory at call time: engines that own
// the whole device through a pre-sized memory pool, code running where an
// allocation would synchronise the device or break a latency budget, and
// hosts whose allocator is not the CUDA runtime's. This entry point serves
// them. The caller passes the image, the source list and the output rows;
// the only other device memory the call needs (the device copy of the
// source list and a status word) is a fixed array defined below, which every
// GPU that loads the library holds until the process exits.
//
// Limits and sharing:
//  - at most GAPSP_NOALLOC_MAX_SOURCES sources per call;
//  - every call uses the same array, which keeps the last call's contents,
//    so calls that overlap on the GPU (different streams, or different host
//    threads with no ordering between them) race: order them on one stream;
//  - the first call on a device looks up the array's device address on that
//    device (the device current at the call); make that first call before
//    any stream capture;
//  - every call waits for its stream: it returns when the rows are complete.
#include <cstring>
#include <mutex>

#include "gapsp.h"
#include "common.cuh"
#include "internal.h"

using namespace gapsp;

namespace {

constexpr size_t kScratchBytes = (size_t)GAPSP_NOALLOC_MAX_SOURCES * sizeof(int32_t) + 256;

// [0, 4 * MAX): the source list; then the status word.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
int32_t g_host_sources[GAPSP_NOALLOC_MAX_SOURCES];  // host staging for validation (under g_mu)

// Device address of the scratch array on the current device, looked up once
// per device: the array's name in host code is not a device address.
gapsp_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return GAPSP_E_CUDA;
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GAPSP_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GAPSP_OK;
}

}  // namespace

extern "C" gapsp_status gapsp_rows_noalloc(const uint8_t* img, int H, int W, int conn, gapsp_kind kind,
                                           const int32_t* sources, int K, uint32_t* out, void* stream) {
    if (H < 1 || W < 1 || H > GAPSP_MAX_SIDE || W > GAPSP_MAX_SIDE || H * W > GAPSP_MAX_N) return GAPSP_E_INVALID;
    if (conn != 4 && conn != 8) return GAPSP_E_INVALID;
    if (kind != GAPSP_GREY && kind != GAPSP_MASK && kind != GAPSP_L1) return GAPSP_E_INVALID;
    if (K < 0 || K > GAPSP_NOALLOC_MAX_SOURCES) return GAPSP_E_INVALID;
    if (K == 0) return GAPSP_OK;
    if (!img || !sources || !out) return GAPSP_E_INVALID;
    if (reinterpret_cast<uintptr_t>(out) & 15) return GAPSP_E_INVALID;  // 16-byte row stores
    // the kernels address the image and the rows directly
    if (!is_device_ptr(img) || !is_device_ptr(out)) return GAPSP_E_INVALID;
    const int N = H * W;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mu);
    void* base = nullptr;
    gapsp_status gs = scratch_address(&base);
    if (gs != GAPSP_OK) return gs;
    int32_t* dsrc = reinterpret_cast<int32_t*>(base);
    int* dstatus = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(base) +
                                          (size_t)GAPSP_NOALLOC_MAX_SOURCES * sizeof(int32_t));
    // validate the sources on the host before anything is written
    if (cudaMemcpyAsync(g_host_sources, sources, (size_t)K * sizeof(int32_t), cudaMemcpyDefault, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    for (int k = 0; k < K; ++k)
        if (g_host_sources[k] < 0 || g_host_sources[k] >= N) return GAPSP_E_INVALID;
    if (cudaMemcpyAsync(dsrc, g_host_sources, (size_t)K * sizeof(int32_t), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(dstatus, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    PropArgs a{};
    a.H = H;
    a.W = W;
    a.N = N;
    a.conn = conn;
    a.kind_mask = kind == GAPSP_MASK;
    a.level_bytes = 1;
    a.f = img;
    a.status = dstatus;
    a.max_sweeps = 4 * (N + 2);
    a.map_base = reinterpret_cast<int*>(out);
    a.sources = dsrc;
    a.njobs = K;
    a.convert = kind == GAPSP_MASK;
    a.phases = K > 304 ? 1 : 4;
    a.cluster = 1;
    if (launch_propagate(a, conn, (int)kind, K, 1, st) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    int sw = 0;
    if (cudaMemcpyAsync(&sw, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return GAPSP_E_CUDA;
    }
    return status_from_word(sw);
}
