// mpn_propagate_noalloc: distances for one grid without allocating anything.
//
// Some callers cannot allocate device memory at all: code running inside
// another framework's memory pool or a fixed-budget allocator, a process that
// must not grow its footprint after start-up, or a real-time loop in which an
// allocation (and the synchronisation it implies) is not allowed. They pass
// their own input and output buffers; every piece of scratch this path needs
// lives in one file-scope device array of fixed size instead.
//
// That array belongs to every GPU that loads this library, from load until the
// process exits (about 2.6 MB). Calls share it and it keeps the last call's
// contents, so each call clears what must start at zero, and two calls whose
// GPU work overlaps (different streams, or different host threads) race on it.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "mpn_internal.cuh"

namespace mpn {
namespace {

// Largest grid this entry point serves: 2048 x 2048 cells.
constexpr int kNaMaxSide = 2048;
constexpr size_t kNaPlaneWords = (size_t)kNaMaxSide * (kNaMaxSide / 32);   // H * P at the limit
constexpr size_t kNaMaxTiles = 1024;
// Tiling used here: compiled variant 0 (128-row x 8-word region), depth 32.
constexpr int kNaVariant = 0;
constexpr int kNaDepth = 32;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaPlaneBytes = align256(kNaPlaneWords * sizeof(uint32_t));
constexpr size_t kNaTileBytes = align256(kNaMaxTiles * 4 * sizeof(uint32_t));
constexpr size_t kNaCtlBytes = align256(sizeof(Ctl));
constexpr size_t kNaScratchBytes = 5 * kNaPlaneBytes + kNaTileBytes + kNaCtlBytes;

// The scratch: free bits, the propagation state (four words per plane word),
// the tile queue, the control block. In host code this name is only a stand-in for the
// device array; the kernels get the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char *g_addr[kMaxDevices] = {};   // device address of the scratch, per device

// Once per device, with that device current: look up the array's address.
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace mpn

using namespace mpn;

extern "C" mpn_status mpn_propagate_noalloc(const uint8_t *mask, int32_t H, int32_t W,
                                            const uint32_t *targets, int32_t n_targets,
                                            uint32_t max_layers, uint32_t *dist, void *stream) {
    if (!mask || !targets || !dist || n_targets < 1) return MPN_EINVAL;
    if (H < 1 || W < 1 || H > kNaMaxSide || W > kNaMaxSide) return MPN_EINVAL;
    const int P = (((W + 31) / 32) + 3) / 4 * 4;
    if ((size_t)H * P > kNaPlaneWords) return MPN_EINVAL;
    const VariantDesc vd = variant_desc(kNaVariant);
    const int ry = region_rows(vd);
    const int TY = ry - 2 * kNaDepth, TXW = vd.rxw - 2;
    const int ntx = ((W + 31) / 32 + TXW - 1) / TXW, nty = (H + TY - 1) / TY;
    const size_t ntiles = (size_t)ntx * nty;
    if (ntiles > kNaMaxTiles) return MPN_EINVAL;

    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return MPN_ECUDA;
    int dev = 0, sms = 0, bps = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = propagate_blocks_per_sm(kNaVariant, 32, &bps);
    if (e != cudaSuccess || bps < 1) return MPN_ECUDA;

    uint32_t *free_bits = reinterpret_cast<uint32_t *>(base);
    uint32_t *state = reinterpret_cast<uint32_t *>(base + kNaPlaneBytes);
    uint32_t *tiles = reinterpret_cast<uint32_t *>(base + 5 * kNaPlaneBytes);
    Ctl *ctl = reinterpret_cast<Ctl *>(base + 5 * kNaPlaneBytes + kNaTileBytes);
    const size_t plane_bytes = (size_t)H * P * sizeof(uint32_t);

    // what must start at zero (the array keeps the previous call's contents)
    e = cudaMemsetAsync(state, 0, 4 * plane_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tiles, 0, ntiles * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dist, 0xff, (size_t)H * W * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = launch_pack(mask, H, W, P, free_bits, st);
    if (e != cudaSuccess) return MPN_ECUDA;

    PropParams p{};
    p.g.free_bits = free_bits;
    p.g.state = state;
    p.g.dist = dist;
    p.g.H = H;
    p.g.W = W;
    p.g.P = P;
    p.queued = tiles;
    p.lists = tiles + ntiles;
    p.ctl = ctl;
    p.ntx = ntx;
    p.nty = nty;
    p.k = kNaDepth;
    p.TY = TY;
    p.TXW = TXW;
    p.max_layers = max_layers;
    p.spin_limit = 1u << 24;
    const uint64_t bound = (max_layers ? (uint64_t)max_layers : (uint64_t)H * W) / kNaDepth + 3;
    p.sweep_cap = (uint32_t)(bound < (1u << 22) ? bound : (1u << 22));
    long long blocks = (long long)bps * sms;
    if (blocks > (long long)ntiles) blocks = (long long)ntiles;
    e = launch_seed(targets, n_targets, p, 32, st);
    if (e == cudaSuccess) e = launch_propagate(kNaVariant, 32, p, (int)blocks, st);
    if (e != cudaSuccess) return MPN_ECUDA;

    // report what the GPU found (bad targets, a timed-out wait)
    uint32_t err = 0;
    e = cudaMemcpyAsync(&err, &ctl->err, sizeof(err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return MPN_ECUDA;
    if (err & ERR_INVAL) return MPN_EINVAL;
    if (err & ERR_OBSTACLE) return MPN_EOBSTACLE;
    if (err & (ERR_TIMEOUT | ERR_SWEEPS)) return MPN_ETIMEOUT;
    return err ? MPN_ECUDA : MPN_OK;
}
