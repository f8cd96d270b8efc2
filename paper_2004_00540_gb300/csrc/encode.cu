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

// Fast path, pass 1: the mask as one flat byte stream (no row structure, so
// every load is an aligned 16-byte vector), packed into a flat bit stream:
// bit f of flat word f / 32 is cell f (row-major), 1 = free; bits past the
// last cell are 0. A lane turns 16 bytes into 16 bits (a byte compare per
// four bytes, the four compare MSBs gathered with one multiply), two lanes
// make a word. Needs a 16-byte-aligned mask.
__global__ void k_pack_flat(const uint8_t *__restrict__ mask, size_t n, uint32_t *__restrict__ flat) {
    const int lane = threadIdx.x & 31;
    const size_t nwords = (n + 31) / 32;
    const size_t chunks = (n + 511) / 512;   // 512 cells per warp and step
    const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t c = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < chunks; c += warps) {
        const size_t b0 = c * 512 + (size_t)lane * 16;
        uint32_t m16 = 0u;
        if (b0 + 16 <= n) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(mask + b0));
            const uint32_t q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t f = __vcmpeq4(q[k], 0u) & 0x80808080u;   // 0x80 per zero byte
                m16 |= ((f * 0x00204081u) >> 28) << (4 * k);
            }
        } else {
            for (int k = 0; k < 16; ++k)
                if (b0 + k < n && mask[b0 + k] == 0) m16 |= 1u << k;
        }
        const uint32_t hi = __shfl_down_sync(0xffffffffu, m16, 1);
        const size_t wi = c * 16 + (size_t)(lane >> 1);
        if (!(lane & 1) && wi < nwords) flat[wi] = m16 | (hi << 16);
    }
}

// Fast path, pass 2: each word of the pitched plane is a 32-bit window of the
// flat bit stream starting at bit y * W + 32 * w (a funnel shift of two flat
// words); bits at x >= W and words past the row are 0.
__global__ void k_pack_rows(const uint32_t *__restrict__ flat, size_t nwords, int H, int W, int P,
                            uint32_t *__restrict__ out) {
    const size_t total = (size_t)H * P;
    auto word = [&](int y, int w) {
        uint32_t v = 0u;
        const int rem = W - w * 32;
        if (rem > 0) {
            const size_t b = (size_t)y * W + (size_t)w * 32;
            const size_t k = b >> 5;
            const uint32_t lo = flat[k], hi = (k + 1 < nwords) ? flat[k + 1] : 0u;
            v = __funnelshift_r(lo, hi, (uint32_t)(b & 31));
            if (rem < 32) v &= (1u << rem) - 1u;
        }
        return v;
    };
    // 32-bit index arithmetic (the usual case) where i + the stride cannot wrap
    if (total + (size_t)gridDim.x * blockDim.x <= 0xffffffffull) {
        const uint32_t t32 = (uint32_t)total, up = (uint32_t)P;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < t32; i += gridDim.x * blockDim.x) {
            const uint32_t y = i / up;
            out[i] = word((int)y, (int)(i - y * up));
        }
        return;
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = word((int)(i / P), (int)(i % P));
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

cudaError_t launch_pack_fast(const uint8_t *mask, int H, int W, int P, uint32_t *free_bits,
                             uint32_t *scratch, size_t scratch_words, cudaStream_t st) {
    const size_t n = (size_t)H * W;
    const size_t nwords = (n + 31) / 32;
    if (((uintptr_t)mask & 15u) || !scratch || scratch_words < nwords)
        return launch_pack(mask, H, W, P, free_bits, st);
    count_launch(2);
    k_pack_flat<<<grid_for((n + 511) / 512, 8), 256, 0, st>>>(mask, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pack_rows<<<grid_for((size_t)H * P, 256), 256, 0, st>>>(scratch, nwords, H, W, P, free_bits);
    return cudaGetLastError();
}

cudaError_t launch_repack(const uint32_t *src, int H, int W, int src_pitch, int P,
                          uint32_t *free_bits, cudaStream_t st) {
    count_launch();
    k_repack<<<grid_for((size_t)H * P, 256), 256, 0, st>>>(src, H, W, src_pitch, P, free_bits);
    return cudaGetLastError();
}

}  // namespace mpn
