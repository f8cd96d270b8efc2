// Encoding of the environment map (Methods, "Input": I_e is 0 on free cells
// and -maxint on obstacles) as one bit per cell: 1 = free. Bit b of word w in
// row y is cell x = 32 * w + b; rows are P words apart; bits at x >= W are 0.
#include <cuda_runtime.h>

#include "mpn_internal.cuh"

namespace mpn {

namespace {

constexpr int kWordsPerWarp = 16;   // one warp packs 16 consecutive words (512 cells)

// mask: H*W uint8, nonzero = obstacle. Each lane reads one byte of each of the
// 16 words (coalesced 32-byte rows of loads), a ballot turns 32 bytes into a
// word, and lanes 0..15 store the 16 words (64 contiguous bytes).
__global__ void k_pack(const uint8_t *__restrict__ mask, int H, int W, int P,
                       uint32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int groups = (P + kWordsPerWarp - 1) / kWordsPerWarp;
    const size_t items = (size_t)H * groups;
    const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t it = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items;
         it += warps) {
        const int y = (int)(it / groups);
        const int w0 = (int)(it % groups) * kWordsPerWarp;
        const uint8_t *row = mask + (size_t)y * W;
        uint8_t v[kWordsPerWarp];
#pragma unroll
        for (int j = 0; j < kWordsPerWarp; ++j) {
            const int x = (w0 + j) * 32 + lane;
            v[j] = (x < W) ? __ldg(row + x) : (uint8_t)1;
        }
        uint32_t mine = 0u;
#pragma unroll
        for (int j = 0; j < kWordsPerWarp; ++j) {
            const uint32_t word = __ballot_sync(0xffffffffu, v[j] == 0);
            if (lane == j) mine = word;
        }
        if (lane < kWordsPerWarp && w0 + lane < P) out[(size_t)y * P + w0 + lane] = mine;
    }
}

// Copy a caller's packed free-cell plane (any pitch) into the context's
// layout, clearing bits at x >= W and words past the row.
__global__ void k_repack(const uint32_t *__restrict__ src, int H, int W, int sp, int P,
                         uint32_t *__restrict__ out) {
    const size_t n = (size_t)H * P;
    const int wv = (W + 31) / 32;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / P), w = (int)(i % P);
        uint32_t v = 0u;
        if (w < wv) {
            v = src[(size_t)y * sp + w];
            const int rem = W - w * 32;
            if (rem < 32) v &= (1u << rem) - 1u;
        }
        out[i] = v;
    }
}

int grid_for(size_t work_items, int per_block) {
    size_t b = (work_items + per_block - 1) / per_block;
    if (b > (size_t)152 * 32) b = (size_t)152 * 32;
    return (int)(b ? b : 1);
}

}  // namespace

cudaError_t launch_pack(const uint8_t *mask, int H, int W, int P, uint32_t *free_bits,
                        cudaStream_t st) {
    const size_t items = (size_t)H * ((P + kWordsPerWarp - 1) / kWordsPerWarp);
    count_launch();
    k_pack<<<grid_for(items, 8), 256, 0, st>>>(mask, H, W, P, free_bits);
    return cudaGetLastError();
}

cudaError_t launch_repack(const uint32_t *src, int H, int W, int src_pitch, int P,
                          uint32_t *free_bits, cudaStream_t st) {
    count_launch();
    k_repack<<<grid_for((size_t)H * P, 256), 256, 0, st>>>(src, H, W, src_pitch, P, free_bits);
    return cudaGetLastError();
}

}  // namespace mpn
