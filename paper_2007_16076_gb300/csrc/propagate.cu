// Kernel (a): host side of the geodesic propagation (the kernels are in
// propagate.cuh, instantiated one edge-cost kind per translation unit so
// that they compile in parallel), and the per-image set-up kernels.
#include "propagate.cuh"

namespace gapsp {

int prop_blocks_per_job(const PropArgs& a) {
    const int C = strips_per_job(a);
    return C > 0 ? C : 1;
}

bool prop_map_in_smem(const PropArgs& a) { return strips_per_job(a) > 0; }

int prop_vpl(int side) {
    if (side <= 32) return 1;
    if (side <= 64) return 2;
    if (side <= 128) return 4;
    if (side <= 256) return 8;
    return -1;
}

cudaError_t launch_propagate(const PropArgs& a, int conn, int kind, int grid, int wpb, cudaStream_t st) {
    const int vpl = prop_vpl(a.H > a.W ? a.H : a.W);
    const int jobs = grid * wpb;  // one block per job
    if (jobs <= 0) return cudaSuccess;
    switch (kind) {
        case 0: return launch_k0(a, conn, vpl, jobs, st);
        case 1: return launch_k1(a, conn, vpl, jobs, st);
        case 2: return launch_k2(a, conn, vpl, jobs, st);
        case 3: return launch_k3(a, conn, vpl, jobs, st);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Per-image set-up: tile geometry of the pixels and boundary flags.
// ---------------------------------------------------------------------------

namespace {

// The 8x8 tile and the bit inside it of every pixel, and the top-left pixel
// of every tile, so that the tree and fill kernels need no division.
__global__ void k_geometry(ImagePrep p) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < p.H * p.W) {
        const int r = q / p.W, c = q - r * p.W;
        p.pgeo[q] = ((uint32_t)((r >> 3) * p.tiles_w + (c >> 3)) << 8) | (uint32_t)(((r & 7) << 3) | (c & 7));
    }
    if (q < p.tiles) {
        const int tr = q / p.tiles_w, tc = q - tr * p.tiles_w;
        p.tbase[q] = (tr << 3) * p.W + (tc << 3);
    }
}

// Boundary vertices: free pixels with fewer free neighbours than the
// connectivity (the image edges on a full grid; Sec. 3.3 and Sec. 5).
__global__ void k_boundary(ImagePrep p) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int N = p.H * p.W;
    if (q >= N) return;
    int r = q / p.W, c = q - r * p.W;
    bool fr = p.kind != 1 || p.f[q];
    int n = 0;
    for (int dr = -1; dr <= 1; ++dr)
        for (int dc = -1; dc <= 1; ++dc) {
            if (!dr && !dc) continue;
            if (p.conn == 4 && dr && dc) continue;
            int rr = r + dr, cc = c + dc;
            if (rr < 0 || rr >= p.H || cc < 0 || cc >= p.W) continue;
            if (p.kind == 1 && !p.f[rr * p.W + cc]) continue;
            ++n;
        }
    p.bound[q] = (fr && n < p.conn) ? 1 : 0;
}

// Levels of a multichannel image for the sum pseudo-metric: F(p) = sum of
// its L channel values (planes of N bytes, channel after channel).
__global__ void k_channel_sum(const uint8_t* planes, int L, int N, uint16_t* F) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int sum = 0;
    for (int l = 0; l < L; ++l) sum += planes[(size_t)l * N + p];
    F[p] = (uint16_t)sum;
}

__global__ void k_unreach(uint32_t* rows, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride)
        if ((int)rows[i] >= PINF) rows[i] = UNREACH;
}

}  // namespace

cudaError_t launch_image_prep(const ImagePrep& p, cudaStream_t st) {
    int N = p.H * p.W;
    k_geometry<<<(N + 255) / 256, 256, 0, st>>>(p);
    k_boundary<<<(N + 255) / 256, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_channel_sum(const uint8_t* planes, int L, int N, uint16_t* F, cudaStream_t st) {
    k_channel_sum<<<(N + 255) / 256, 256, 0, st>>>(planes, L, N, F);
    return cudaGetLastError();
}

cudaError_t launch_unreach_convert(uint32_t* rows, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_unreach<<<1216, 256, 0, st>>>(rows, n);
    return cudaGetLastError();
}

}  // namespace gapsp
