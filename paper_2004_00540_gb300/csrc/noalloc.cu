// mpn_propagate_noalloc: distances for one grid without allocating anything.
//
// Some callers cannot allocate device memory at all: code running inside
// another framework's memory pool or a fixed-budget allocator, a process that
// must not grow its footprint after start-up, or a real-time loop in which an
// allocation (and the synchronisation it implies) is not allowed. They pass
// their own input and output buffers; every piece of scratch this path needs
// lives in one file-scope device array of fixed size instead.
//
// That array (about 2.6 MB) belongs to every GPU on which this library's
// device code is loaded, until the process exits. With lazy module loading
// (the CUDA default) the code and the array are loaded on a device at the
// first use, which for a caller of this entry point alone is its first call
// there (the address lookup below): that call, or a warm-up call made at
// start-up, is when the footprint grows. Calls share the array and it keeps
// the last call's contents, so each call clears what must start at zero, and
// two calls whose GPU work overlaps (different streams, or different host
// threads) race on it.
#include <cstring>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

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
constexpr size_t kNaTileBytes = align256((kRankWords + kTileQueueWords * kNaMaxTiles + 3) / 4 * 4 * sizeof(uint32_t));
constexpr size_t kNaCtlBytes = align256(sizeof(Ctl));
constexpr size_t kNaScratchBytes = 5 * kNaPlaneBytes + kNaTileBytes + kNaCtlBytes;

// The scratch: free bits, the propagation state (four words per plane word),
// the tile queue, the control block. In host code this name is only a stand-in for the
// device array; the kernels get the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
// Device address of the scratch, per device, with the id of the context it
// was looked up in: a device reset ends that context and the array comes back
// at a new address in the next one, so the lookup is repeated when the
// current context's id (unique for the life of the process) changes.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    unsigned char *addr = nullptr;
};
ScratchAddr g_addr[kMaxDevices];

template <typename F>
F driver_fn(const char *name, int version) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return (F)f;
    cudaGetLastError();
    return nullptr;
}

// id of the current context; 0 when there is none yet
bool current_ctx_id(unsigned long long *id) {
    static PFN_cuCtxGetCurrent_v4000 get_ctx = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        get_ctx = driver_fn<PFN_cuCtxGetCurrent_v4000>("cuCtxGetCurrent", 4000);
        get_id = driver_fn<PFN_cuCtxGetId_v12000>("cuCtxGetId", 12000);
    });
    if (!get_ctx || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) return false;
    *id = 0;
    return !ctx || get_id(ctx, id) == CUDA_SUCCESS;
}

// Set-up, once per device (and again after a reset of it), with that device
// current: look up the array's device address. In host code the array's name
// is only a stand-in; kernels must get this address.
cudaError_t scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;   // 0: the runtime has not set the device up yet
    if (!current_ctx_id(&id)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr &a = g_addr[dev];
    if (!id || a.ctx_id != id || !a.addr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // sets the context up if needed
        if (e != cudaSuccess) return e;
        if (!id && (!current_ctx_id(&id) || !id)) return cudaErrorDeviceUninitialized;
        a.ctx_id = id;
        a.addr = static_cast<unsigned char *>(p);
    }
    *out = a.addr;
    return cudaSuccess;
}

// Device memory of device `dev` (device or managed allocation), read in place
// by the kernels. Allocates nothing.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
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
    int dev = 0, sms = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return MPN_ECUDA;
    // the kernels read and write these in place: all three must be memory of
    // the current device
    if (!on_device(mask, dev) || !on_device(targets, dev) || !on_device(dist, dev))
        return MPN_EINVAL;
    unsigned char *base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return MPN_ECUDA;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = propagate_blocks_per_sm(kNaVariant, 32, &bps);
    if (e != cudaSuccess || bps < 1) return MPN_ECUDA;

    uint32_t *free_bits = reinterpret_cast<uint32_t *>(base);
    uint32_t *state = reinterpret_cast<uint32_t *>(base + kNaPlaneBytes);
    uint32_t *tiles = reinterpret_cast<uint32_t *>(base + 5 * kNaPlaneBytes);
    Ctl *ctl = reinterpret_cast<Ctl *>(base + 5 * kNaPlaneBytes + kNaTileBytes);
    const size_t plane_bytes = (size_t)H * P * sizeof(uint32_t);

    // what must start at zero (the array keeps the previous call's contents)
    PropParams p{};
    size_t clear_words = 0;
    layout_tile_queue(tiles, ntiles, false, &p, &clear_words);
    e = cudaMemsetAsync(state, 0, 4 * plane_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tiles, 0, clear_words * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dist, 0xff, (size_t)H * W * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = launch_pack(mask, H, W, P, free_bits, st);
    if (e != cudaSuccess) return MPN_ECUDA;

    p.g.free_bits = free_bits;
    p.g.state = state;
    p.g.dist = dist;
    p.g.H = H;
    p.g.W = W;
    p.g.P = P;
    p.ctl = ctl;
    p.ntx = ntx;
    p.nty = nty;
    p.k = kNaDepth;
    p.TY = TY;
    p.TXW = TXW;
    p.max_layers = max_layers;
    p.spin_limit = 1u << 24;
    p.lookahead = 1;
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
