// C ABI of the max-pooling path planner: context, device memory, staging of
// host arguments, stream ordering and error reporting. Every entry point is
// declared and documented in include/mpn.h.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include <cuda_runtime.h>

#include "mpn_internal.cuh"

using namespace mpn;

namespace {

std::atomic<uint64_t> g_launches{0};

constexpr uint32_t kSpinLimit = 1u << 24;   // ~ seconds of 100 ns polls

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want) {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mpn_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return MPN_OK;
    mpn::note_cuda_error(e);
    if (e == cudaErrorMemoryAllocation) return MPN_ENOMEM;
    return MPN_ECUDA;
}

mpn_status from_err_bits(uint32_t e) {
    if (!e) return MPN_OK;
    if (e & ERR_INVAL) return MPN_EINVAL;
    if (e & ERR_OBSTACLE) return MPN_EOBSTACLE;
    if (e & ERR_OVERFLOW) return MPN_EOVERFLOW;
    if (e & (ERR_TIMEOUT | ERR_SWEEPS)) return MPN_ETIMEOUT;
    return MPN_ECUDA;
}

#define MPN_TRY(expr)                                   \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return from_cuda(e_);    \
    } while (0)

}  // namespace

namespace mpn {
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

thread_local cudaError_t g_last_error = cudaSuccess;
void note_cuda_error(cudaError_t e) { g_last_error = e; }

// Autotuner table: per size bucket, the fastest depth measured for each tile
// shape and the fastest (shape, depth) overall.
namespace {
constexpr int kBuckets = 33, kMaxVariants = 16;
struct TuneTable {
    std::mutex mu;
    int depth[kBuckets][kMaxVariants] = {};
    float ms[kBuckets][kMaxVariants] = {};
    int best_v[kBuckets], best_d[kBuckets] = {};
    float best_ms[kBuckets] = {};
    TuneTable() {
        for (int b = 0; b < kBuckets; ++b) best_v[b] = -1;
    }
};
TuneTable g_tune;

int bucket_of(int H, int W) {
    int m = H > W ? H : W, b = 0;
    while ((1 << b) < m && b < kBuckets - 1) ++b;
    return b;
}
}  // namespace

bool tune_lookup(int H, int W, int variant, int *depth) {
    if (variant < 0 || variant >= kMaxVariants) return false;
    std::lock_guard<std::mutex> lk(g_tune.mu);
    const int b = bucket_of(H, W);
    if (!g_tune.depth[b][variant]) return false;
    *depth = g_tune.depth[b][variant];
    return true;
}

bool tune_best(int H, int W, int *variant, int *depth) {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    const int b = bucket_of(H, W);
    if (g_tune.best_v[b] < 0) return false;
    *variant = g_tune.best_v[b];
    *depth = g_tune.best_d[b];
    return true;
}

static void tune_record(int H, int W, int variant, int depth, float ms) {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    const int b = bucket_of(H, W);
    if (!g_tune.depth[b][variant] || ms < g_tune.ms[b][variant]) {
        g_tune.depth[b][variant] = depth;
        g_tune.ms[b][variant] = ms;
    }
    if (g_tune.best_v[b] < 0 || ms < g_tune.best_ms[b]) {
        g_tune.best_v[b] = variant;
        g_tune.best_d[b] = depth;
        g_tune.best_ms[b] = ms;
    }
}
}  // namespace mpn

struct mpn_ctx {
    int H = 0, W = 0, P = 0, dist_bits = 32;
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;

    DevBuf free_bits, state, dist, ctl, tiles, mask_stage, log;
    DevBuf targets, starts, offsets, status, cells, activity, order;
    DevBuf jump, segs;   // long walks: jump table (2 * H * W words), segments + counter
    DevBuf check;        // violation counter of mpn_check

    int variant = 0, depth = 32;
    bool auto_tune = true;
    int ntx = 0, nty = 0, TY = 0, TXW = 0, blocks = 0;

    bool propagated = false;
    uint32_t last_layers = 0, last_max_layers = 0;
    bool stats_pending = false;
    Ctl last_ctl{};

    // page-locked, device-mapped host words that small results (the control
    // block, a path total, an error word) are stored to by k_store_host
    unsigned char *mbox = nullptr, *mbox_d = nullptr;

    cudaEvent_t ev[6] = {};   // encode begin/end, propagate begin/end, trace begin/end
    float ms_encode = 0.f, ms_propagate = 0.f, ms_trace = 0.f;
    bool ev_enc = false, ev_prop = false, ev_trace = false;
    // asynchronous distance copy: ev_ready orders it after the context's
    // stream, ev_out marks its end on the copy's stream
    cudaEvent_t ev_ready = nullptr, ev_out = nullptr;
    bool out_pending = false;

    GridDev grid() const {
        GridDev g;
        g.free_bits = (const uint32_t *)free_bits.p;
        g.state = (uint32_t *)state.p;
        g.dist = dist.p;
        g.H = H;
        g.W = W;
        g.P = P;
        return g;
    }
    size_t plane_words() const { return (size_t)H * P; }
    size_t dist_bytes() const { return (size_t)H * W * (dist_bits / 8); }
};

namespace mpn {

// Device-to-host copy by SM stores over the coherent CPU-GPU link rather than
// a copy engine. Device-to-host copy-engine transfers run in the order they
// were issued, across streams, so a small read-back on one context's stream
// would otherwise wait for a large distance download that another context
// started first; stores from a kernel do not queue behind it.
__global__ void k_store_host(const unsigned char *__restrict__ src, unsigned char *__restrict__ dst,
                             size_t bytes) {
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t nt = (size_t)gridDim.x * blockDim.x;
    const uintptr_t a = (uintptr_t)src | (uintptr_t)dst;
    size_t done = 0;
    if ((a & 15) == 0) {
        const size_t nv = bytes / 16;
        for (size_t i = t0; i < nv; i += nt) ((uint4 *)dst)[i] = ((const uint4 *)src)[i];
        done = nv * 16;
    } else if ((a & 3) == 0) {
        const size_t nv = bytes / 4;
        for (size_t i = t0; i < nv; i += nt) ((uint32_t *)dst)[i] = ((const uint32_t *)src)[i];
        done = nv * 4;
    }
    for (size_t i = done + t0; i < bytes; i += nt) dst[i] = src[i];
}

}  // namespace mpn

namespace {

// Mailbox layout (bytes): the control block, then a path total and an error word.
constexpr size_t kMboxCtl = 0, kMboxTotal = 128, kMboxErr = 136, kMboxWalk = 140, kMboxCheck = 144,
                 kMboxBytes = 256;
static_assert(sizeof(Ctl) <= kMboxTotal, "control block must fit the mailbox");

cudaError_t store_host(mpn_ctx *c, void *dst_dev, const void *src, size_t bytes) {
    if (!bytes) return cudaSuccess;
    const size_t per_block = 256 * 16 * 4;
    const size_t want = (bytes + per_block - 1) / per_block;
    const int blocks = (int)(want < (size_t)c->sm_count ? (want ? want : 1) : (size_t)c->sm_count);
    k_store_host<<<blocks, 256, 0, c->stream>>>((const unsigned char *)src, (unsigned char *)dst_dev,
                                                bytes);
    count_launch();
    return cudaGetLastError();
}

// The device address of page-locked host memory, else null (device memory,
// or pageable host memory).
void *pinned_devptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Copy a device result to the caller's buffer, ordered on the context's
// stream: device memory by a device-to-device copy, page-locked host memory by
// k_store_host, pageable host memory by a copy engine.
cudaError_t copy_out(mpn_ctx *c, void *dst, const void *src, size_t bytes) {
    if (!bytes) return cudaSuccess;
    if (is_device_ptr(dst)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (void *d = pinned_devptr(dst)) return store_host(c, d, src, bytes);
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
}

// Store device bytes into the context's mailbox at offset off (read on the
// host after the stream is synchronized).
cudaError_t to_mbox(mpn_ctx *c, size_t off, const void *src, size_t bytes) {
    return store_host(c, c->mbox_d + off, src, bytes);
}

// Tile geometry and grid size for (variant, depth); allocates the tile queue
// (per tile a stamp, the latest log header and the logged-visit count, three
// tile lists, then the per-tile header slots).
mpn_status configure(mpn_ctx *c, int variant, int depth) {
    if (variant < 0 || variant >= num_variants()) return MPN_EINVAL;
    const VariantDesc vd = variant_desc(variant);
    const int ry = region_rows(vd);
    // the halo (depth rows) must not reach past the neighbouring tiles: a
    // visit queues only its 8 neighbours, so the interior needs >= depth rows
    if (depth < 1 || depth > 32 || ry - 2 * depth < depth) return MPN_EINVAL;
    const int TY = ry - 2 * depth, TXW = vd.rxw - 2;
    const int wwords = (c->W + 31) / 32;
    const int ntx = (wwords + TXW - 1) / TXW, nty = (c->H + TY - 1) / TY;
    if (vd.tma && c->dist_bits != 32) return MPN_EINVAL;   // the TMA shape writes uint32 planes
    int bps = 0;
    MPN_TRY(propagate_blocks_per_sm(variant, c->dist_bits, &bps));
    if (bps < 1) return MPN_ECUDA;
    const long long ntiles = (long long)ntx * nty;
    long long blocks = (long long)bps * c->sm_count;
    if (blocks > ntiles) blocks = ntiles;
    if (blocks < 1) blocks = 1;
    MPN_TRY(c->tiles.ensure(tile_queue_words((size_t)ntiles, true) * sizeof(uint32_t)));
    c->variant = variant;
    c->depth = depth;
    c->TY = TY;
    c->TXW = TXW;
    c->ntx = ntx;
    c->nty = nty;
    c->blocks = (int)blocks;
    return MPN_OK;
}

// Automatic tiling: the autotuner's choice for this size bucket if one was
// measured, else the 128-row x 256-cell region: for grids up to 2^22 cells
// (few tiles: fewer sweeps matter most) shape 0 at depth 32, above them shape
// 12 (four warps of two words x four rows per lane) at depth 28, the fastest
// measured on a 23170^2 grid.
mpn_status auto_configure(mpn_ctx *c) {
    int v = 0, d = 32;
    if (tune_best(c->H, c->W, &v, &d) && configure(c, v, d) == MPN_OK) return MPN_OK;
    if ((int64_t)c->H * c->W > (1ll << 22)) return configure(c, 12, 28);
    return configure(c, 0, 32);
}

mpn_status alloc_planes(mpn_ctx *c) {
    const size_t pw = c->plane_words() * sizeof(uint32_t);
    MPN_TRY(c->free_bits.ensure(pw));
    MPN_TRY(c->state.ensure(4 * pw));
    MPN_TRY(c->dist.ensure(c->dist_bytes()));
    MPN_TRY(c->ctl.ensure(sizeof(Ctl)));
    for (auto &e : c->ev) MPN_TRY(cudaEventCreate(&e));
    MPN_TRY(cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming));
    MPN_TRY(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    return auto_configure(c);
}

mpn_status new_ctx(int32_t H, int32_t W, int32_t dist_bits, void *stream, mpn_ctx **out) {
    if (!out) return MPN_EINVAL;
    *out = nullptr;
    if (H < 1 || W < 1 || (uint64_t)H * (uint64_t)W >= 0xffffffffull) return MPN_EINVAL;
    if (dist_bits == MPN_DIST_AUTO) dist_bits = ((int64_t)H * W <= 65535) ? 16 : 32;
    if (dist_bits != 16 && dist_bits != 32) return MPN_EINVAL;
    mpn_ctx *c = new (std::nothrow) mpn_ctx();
    if (!c) return MPN_ENOMEM;
    c->H = H;
    c->W = W;
    c->P = (((W + 31) / 32) + 3) / 4 * 4;
    c->dist_bits = dist_bits;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->mbox, kMboxBytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&c->mbox_d, c->mbox, 0);
    if (e != cudaSuccess) {
        if (c->mbox) cudaFreeHost(c->mbox);
        delete c;
        return from_cuda(e);
    }
    mpn_status st = alloc_planes(c);
    if (st != MPN_OK) {
        mpn_destroy(c);
        return st;
    }
    *out = c;
    return MPN_OK;
}

// Copy n uint32 values to a device staging buffer unless already on device.
mpn_status stage_u32(mpn_ctx *c, DevBuf &buf, const uint32_t *src, int32_t n,
                     const uint32_t **dev) {
    if (n <= 0) {
        *dev = nullptr;
        return MPN_OK;
    }
    if (is_device_ptr(src)) {
        *dev = src;
        return MPN_OK;
    }
    MPN_TRY(buf.ensure((size_t)n * sizeof(uint32_t)));
    MPN_TRY(cudaMemcpyAsync(buf.p, src, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            c->stream));
    *dev = (const uint32_t *)buf.p;
    return MPN_OK;
}

mpn_status encode_mask(mpn_ctx *c, const uint8_t *mask) {
    if (!mask) return MPN_EINVAL;
    const uint8_t *dm = mask;
    MPN_TRY(cudaEventRecord(c->ev[0], c->stream));
    if (!is_device_ptr(mask)) {
        const size_t n = (size_t)c->H * c->W;
        MPN_TRY(c->mask_stage.ensure(n));
        MPN_TRY(cudaMemcpyAsync(c->mask_stage.p, mask, n, cudaMemcpyHostToDevice, c->stream));
        dm = (const uint8_t *)c->mask_stage.p;
    }
    // the propagation state is scratch here: every propagate clears it first
    MPN_TRY(launch_pack_fast(dm, c->H, c->W, c->P, (uint32_t *)c->free_bits.p, (uint32_t *)c->state.p,
                             c->state.bytes / sizeof(uint32_t), c->stream));
    MPN_TRY(cudaEventRecord(c->ev[1], c->stream));
    c->ev_enc = true;
    c->propagated = false;
    return MPN_OK;
}

// Collect the device-side result of the last propagate (waits).
mpn_status finish_propagate(mpn_ctx *c) {
    if (!c->stats_pending) return MPN_OK;
    MPN_TRY(to_mbox(c, kMboxCtl, c->ctl.p, sizeof(Ctl)));
    MPN_TRY(cudaStreamSynchronize(c->stream));
    memcpy(&c->last_ctl, c->mbox + kMboxCtl, sizeof(Ctl));
    c->stats_pending = false;
    c->last_layers = c->last_ctl.max_layer;
    if (c->last_ctl.err) {
        c->propagated = false;
        return from_err_bits(c->last_ctl.err);
    }
    return MPN_OK;
}

// fill_dist: set the distance plane to "unreached" first (the per-layer
// kernel and a propagation without the activation log write only the cells
// they reach; the log decode writes every cell).
mpn_status begin_propagate(mpn_ctx *c, const uint32_t *targets, int32_t n,
                           const uint32_t **dt, bool fill_dist) {
    if (!c) return MPN_EINVAL;
    if (!targets || n < 1) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);   // drain an earlier run's error report
    (void)st;
    if (c->out_pending) {   // the plane is rewritten below: after the pending copy
        MPN_TRY(cudaStreamWaitEvent(c->stream, c->ev_out, 0));
        c->out_pending = false;
    }
    c->propagated = false;
    if (!is_device_ptr(targets)) {
        const uint64_t N = (uint64_t)c->H * c->W;
        for (int32_t i = 0; i < n; ++i)
            if ((uint64_t)targets[i] >= N) return MPN_EINVAL;
    }
    st = stage_u32(c, c->targets, targets, n, dt);
    if (st != MPN_OK) return st;
    if (fill_dist) MPN_TRY(cudaMemsetAsync(c->dist.p, 0xff, c->dist_bytes(), c->stream));
    MPN_TRY(cudaMemsetAsync(c->state.p, 0, c->plane_words() * 16, c->stream));
    MPN_TRY(cudaMemsetAsync(c->ctl.p, 0, sizeof(Ctl), c->stream));
    return MPN_OK;
}

}  // namespace

extern "C" {

const char *mpn_status_str(mpn_status s) {
    switch (s) {
        case MPN_OK: return "ok";
        case MPN_EINVAL: return "invalid argument";
        case MPN_ENOMEM: return "out of memory or output capacity too small";
        case MPN_ECUDA: return "CUDA runtime error";
        case MPN_ETIMEOUT: return "grid-wide wait timed out";
        case MPN_EOVERFLOW: return "distance does not fit the uint16 plane";
        case MPN_EOBSTACLE: return "target on an obstacle";
        case MPN_ESTATE: return "call out of order";
        case MPN_ECHECK: return "distance plane fails the invariant check";
    }
    return "unknown status";
}

uint64_t mpn_launch_count(void) { return g_launches.load(); }

const char *mpn_last_error(void) {
    return mpn::g_last_error == cudaSuccess ? "" : cudaGetErrorString(mpn::g_last_error);
}

mpn_status mpn_create(const uint8_t *mask, int32_t H, int32_t W, int32_t dist_bits, void *stream,
                      mpn_ctx **out) {
    NvtxRange nvtx_range("mpn_create");
    if (!mask) return MPN_EINVAL;
    mpn_status st = new_ctx(H, W, dist_bits, stream, out);
    if (st != MPN_OK) return st;
    st = encode_mask(*out, mask);
    if (st != MPN_OK) {
        mpn_destroy(*out);
        *out = nullptr;
    }
    return st;
}

mpn_status mpn_create_packed(const uint32_t *bits, int32_t H, int32_t W, int32_t pitch_words,
                             int32_t dist_bits, void *stream, mpn_ctx **out) {
    if (!bits || pitch_words < (W + 31) / 32) return MPN_EINVAL;
    mpn_status st = new_ctx(H, W, dist_bits, stream, out);
    if (st != MPN_OK) return st;
    mpn_ctx *c = *out;
    const uint32_t *src = bits;
    DevBuf tmp;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(bits)) {
        const size_t bytes = (size_t)H * pitch_words * 4;
        e = tmp.ensure(bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp.p, bits, bytes, cudaMemcpyHostToDevice, c->stream);
        src = (const uint32_t *)tmp.p;
    }
    if (e == cudaSuccess) e = launch_repack(src, H, W, pitch_words, c->P, (uint32_t *)c->free_bits.p, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    tmp.release();
    if (e != cudaSuccess) {
        mpn_destroy(c);
        *out = nullptr;
        return from_cuda(e);
    }
    return MPN_OK;
}

mpn_status mpn_set_mask(mpn_ctx *c, const uint8_t *mask) {
    NvtxRange nvtx_range("mpn_set_mask");
    if (!c) return MPN_EINVAL;
    finish_propagate(c);
    return encode_mask(c, mask);
}

mpn_status mpn_set_stream(mpn_ctx *c, void *stream) {
    if (!c) return MPN_EINVAL;
    c->stream = (cudaStream_t)stream;
    return MPN_OK;
}

mpn_status mpn_set_tuning(mpn_ctx *c, int32_t variant, int32_t depth) {
    if (!c) return MPN_EINVAL;
    if (variant < 0) {
        c->auto_tune = true;
        return auto_configure(c);
    }
    mpn_status st = configure(c, variant, depth);
    if (st == MPN_OK) c->auto_tune = false;
    return st;
}

mpn_status mpn_variant_info(int32_t v, int32_t *rows, int32_t *words, int32_t *threads) {
    if (v < 0 || v >= num_variants()) return MPN_EINVAL;
    const VariantDesc d = variant_desc(v);
    if (rows) *rows = region_rows(d);
    if (words) *words = d.rxw;
    if (threads) *threads = variant_threads(v);
    return MPN_OK;
}

// A run of the persistent kernel (and the log decode) seeded either from
// targets (din null: layer 0 = the targets) or from a distance plane din
// (device, H * W of the dtype; cells at distance <= from are kept).
static mpn_status run_propagate(mpn_ctx *c, const uint32_t *targets, int32_t n, const void *din,
                                uint32_t from, uint32_t max_layers, uint32_t *layers_run) {
    // activation log: room for 1.5 entries per plane word plus one partly
    // filled chunk per block (a block that finds it full writes distances
    // itself, so the size only affects speed). The TMA-staged variant writes
    // its distances itself.
    const uint64_t log_entries = c->plane_words() * 3 / 2 + (uint64_t)c->blocks * kLogChunk;
    // (a visit's header and entries must fit one chunk; every compiled tiling does)
    uint32_t log_chunks = (variant_desc(c->variant).tma || (uint64_t)c->TY * c->TXW + 1 > kLogChunk)
                              ? 0u : (uint32_t)((log_entries + kLogChunk - 1) / kLogChunk);
    // test hooks for the fallback paths: a smaller pool (MPN_TEST_LOG_CHUNKS;
    // 0 = no log), fewer decode slots (MPN_TEST_DECODE_SLOTS)
    if (const char *e = getenv("MPN_TEST_LOG_CHUNKS")) {
        const long v = strtol(e, nullptr, 10);
        if (v >= 0 && (uint64_t)v < log_chunks) log_chunks = (uint32_t)v;
    }
    uint32_t slots = kTileSlots;
    if (const char *e = getenv("MPN_TEST_DECODE_SLOTS")) slots = (uint32_t)strtoul(e, nullptr, 10);
    if (log_chunks &&
        c->log.ensure((size_t)log_chunks * kLogFields * kLogChunk * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();   // no room for the log: the kernel writes distances itself
        c->log.release();
        log_chunks = 0;
    }
    const uint32_t *dt = nullptr;
    mpn_status st = din ? MPN_OK : begin_propagate(c, targets, n, &dt, log_chunks == 0);
    if (st != MPN_OK) return st;
    const size_t ntiles = (size_t)c->ntx * c->nty;
    PropParams p{};
    p.g = c->grid();
    size_t clear_words = 0;
    layout_tile_queue((uint32_t *)c->tiles.p, ntiles, true, &p, &clear_words);
    // queue stamps, done stamps, latest log headers, logged-visit counts, lists
    MPN_TRY(cudaMemsetAsync(c->tiles.p, 0, clear_words * sizeof(uint32_t), c->stream));
    p.ctl = (Ctl *)c->ctl.p;
    p.ntx = c->ntx;
    p.nty = c->nty;
    p.k = c->depth;
    p.TY = c->TY;
    p.TXW = c->TXW;
    p.max_layers = max_layers;
    p.l_base = from;
    p.spin_limit = kSpinLimit;
    p.lookahead = 1;
    // (test hook: MPN_TEST_NO_LOOKAHEAD=1 makes blocks only wait at a sweep's end)
    if (const char *e = getenv("MPN_TEST_NO_LOOKAHEAD")) p.lookahead = (e[0] == '1') ? 0u : 1u;
    p.log = log_chunks ? (uint32_t *)c->log.p : nullptr;
    p.log_chunks = log_chunks;
    const uint64_t bound = (max_layers ? (uint64_t)(max_layers - from) : (uint64_t)c->H * c->W) / c->depth + 3;
    p.sweep_cap = (uint32_t)(bound < (1u << 22) ? bound : (1u << 22));
    // test hooks that make the device-side limits run out on purpose (the
    // kernel then records the error and every block returns):
    // MPN_TEST_SPIN_LIMIT polls per grid-barrier wait, MPN_TEST_SWEEP_CAP sweeps
    if (const char *e = getenv("MPN_TEST_SPIN_LIMIT")) {
        const long v = strtol(e, nullptr, 10);
        if (v >= 0 && (uint64_t)v < p.spin_limit) p.spin_limit = (uint32_t)v;
    }
    if (const char *e = getenv("MPN_TEST_SWEEP_CAP")) {
        const long v = strtol(e, nullptr, 10);
        if (v >= 1 && (uint64_t)v < p.sweep_cap) p.sweep_cap = (uint32_t)v;
    }
    if (din) MPN_TRY(launch_seed_plane(din, p, c->dist_bits, c->stream));
    else MPN_TRY(launch_seed(dt, n, p, c->dist_bits, c->stream));
    MPN_TRY(cudaEventRecord(c->ev[2], c->stream));   // times the persistent kernel + log decode
    MPN_TRY(launch_propagate(c->variant, c->dist_bits, p, c->blocks, c->stream));
    MPN_TRY(launch_log_decode(p, c->dist_bits, c->sm_count, slots, c->stream));
    MPN_TRY(cudaEventRecord(c->ev[3], c->stream));
    c->ev_prop = true;
    c->stats_pending = true;
    c->propagated = true;
    c->last_max_layers = max_layers;
    if (layers_run) {
        st = finish_propagate(c);
        if (st != MPN_OK) return st;
        *layers_run = c->last_layers;
    }
    return MPN_OK;
}

// the invariant check of the context's plane (after its propagation)
static mpn_status check_plane(mpn_ctx *c, uint64_t *violations) {
    MPN_TRY(c->check.ensure(sizeof(unsigned long long)));
    MPN_TRY(launch_check_plane(c->grid(), c->dist_bits, c->last_max_layers,
                               (unsigned long long *)c->check.p, c->stream));
    MPN_TRY(to_mbox(c, kMboxCheck, c->check.p, sizeof(uint64_t)));
    MPN_TRY(cudaStreamSynchronize(c->stream));
    uint64_t v = 0;
    memcpy(&v, c->mbox + kMboxCheck, sizeof(v));
    if (violations) *violations = v;
    return v ? MPN_ECHECK : MPN_OK;
}

static bool check_mode() {
    const char *e = getenv("MPN_CHECK");
    return e && e[0] == '1';
}

mpn_status mpn_propagate(mpn_ctx *c, const uint32_t *targets, int32_t n, uint32_t max_layers,
                         uint32_t *layers_run) {
    NvtxRange nvtx_range("mpn_propagate");
    if (!c || !targets || n < 1) return MPN_EINVAL;
    mpn_status st = run_propagate(c, targets, n, nullptr, 0u, max_layers, layers_run);
    if (st == MPN_OK && layers_run && check_mode()) st = check_plane(c, nullptr);
    return st;
}

mpn_status mpn_check(mpn_ctx *c, uint64_t *violations) {
    NvtxRange nvtx_range("mpn_check");
    if (!c) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    if (st != MPN_OK) return st;
    if (!c->propagated) return MPN_ESTATE;
    return check_plane(c, violations);
}

mpn_status mpn_propagate_resume(mpn_ctx *c, const void *dist_in, uint32_t from_layer,
                                uint32_t max_layers, uint32_t *layers_run) {
    NvtxRange nvtx_range("mpn_propagate_resume");
    if (!c || !dist_in) return MPN_EINVAL;
    if (max_layers && max_layers <= from_layer) return MPN_EINVAL;
    const uint32_t inf = c->dist_bits == 16 ? 0xffffu : 0xffffffffu;
    if (from_layer >= inf) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);   // drain an earlier run's error report
    (void)st;
    if (c->out_pending) {   // the plane is rewritten below: after the pending copy
        MPN_TRY(cudaStreamWaitEvent(c->stream, c->ev_out, 0));
        c->out_pending = false;
    }
    c->propagated = false;
    // the seed reads the plane and writes the context's own plane (in place
    // for a host plane, which goes there first)
    const void *din = dist_in;
    if (!is_device_ptr(dist_in)) {
        MPN_TRY(cudaMemcpyAsync(c->dist.p, dist_in, c->dist_bytes(), cudaMemcpyHostToDevice, c->stream));
        din = c->dist.p;
    }
    MPN_TRY(cudaMemsetAsync(c->state.p, 0, c->plane_words() * 16, c->stream));
    MPN_TRY(cudaMemsetAsync(c->ctl.p, 0, sizeof(Ctl), c->stream));
    return run_propagate(c, nullptr, 0, din, from_layer, max_layers, layers_run);
}

mpn_status mpn_propagate_plain(mpn_ctx *c, const uint32_t *targets, int32_t n,
                               uint32_t max_layers, int32_t check_every, uint32_t *layers_run) {
    if (check_every < 1) return MPN_EINVAL;
    const uint32_t *dt = nullptr;
    mpn_status st = begin_propagate(c, targets, n, &dt, true);
    if (st != MPN_OK) return st;
    Ctl *ctl = (Ctl *)c->ctl.p;
    const GridDev g = c->grid();
    MPN_TRY(cudaEventRecord(c->ev[2], c->stream));
    MPN_TRY(launch_plain_seed(dt, n, g, c->dist_bits, ctl, c->stream));
    uint32_t layer = 1;
    for (;;) {
        for (int q = 0; q < check_every; ++q, ++layer) {
            if (max_layers && layer > max_layers) break;
            MPN_TRY(launch_plain_layer(g, c->dist_bits, layer, ctl, c->stream));
        }
        Ctl h;
        MPN_TRY(to_mbox(c, kMboxCtl, ctl, sizeof(Ctl)));
        MPN_TRY(cudaStreamSynchronize(c->stream));
        memcpy(&h, c->mbox + kMboxCtl, sizeof(Ctl));
        if (h.err) {
            c->propagated = false;
            return from_err_bits(h.err);
        }
        // stop once a layer added nothing, or the fixed depth is reached
        if (h.plain_last + 1 < layer || (max_layers && layer > max_layers)) {
            c->last_layers = h.plain_last;
            break;
        }
    }
    MPN_TRY(cudaEventRecord(c->ev[3], c->stream));
    c->ev_prop = true;
    c->propagated = true;
    c->stats_pending = false;
    c->last_max_layers = max_layers;
    if (layers_run) *layers_run = c->last_layers;
    return MPN_OK;
}

mpn_status mpn_sync(mpn_ctx *c) {
    if (!c) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    if (st != MPN_OK) return st;
    if (c->out_pending) MPN_TRY(cudaEventSynchronize(c->ev_out));
    return from_cuda(cudaStreamSynchronize(c->stream));
}

mpn_status mpn_get_distances(mpn_ctx *c, void *dst, int32_t on_device) {
    NvtxRange nvtx_range("mpn_get_distances");
    if (!c || !dst) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    if (st != MPN_OK) return st;
    if (!c->propagated) return MPN_ESTATE;
    MPN_TRY(cudaMemcpyAsync(dst, c->dist.p, c->dist_bytes(),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->stream));
    return from_cuda(cudaStreamSynchronize(c->stream));
}

mpn_status mpn_get_distances_async(mpn_ctx *c, void *dst, void *stream) {
    if (!c || !dst) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    if (st != MPN_OK) return st;
    if (!c->propagated) return MPN_ESTATE;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    if (s != c->stream) {
        MPN_TRY(cudaEventRecord(c->ev_ready, c->stream));
        MPN_TRY(cudaStreamWaitEvent(s, c->ev_ready, 0));
    }
    MPN_TRY(cudaMemcpyAsync(dst, c->dist.p, c->dist_bytes(), cudaMemcpyDefault, s));
    MPN_TRY(cudaEventRecord(c->ev_out, s));
    c->out_pending = true;
    return MPN_OK;
}

mpn_status mpn_get_activity(mpn_ctx *c, uint32_t L, int32_t *dst, int32_t on_device) {
    if (!c || !dst) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    if (st != MPN_OK) return st;
    if (!c->propagated) return MPN_ESTATE;
    if (L == 0) L = c->last_layers;
    const size_t bytes = (size_t)c->H * c->W * sizeof(int32_t);
    int32_t *out = dst;
    if (!on_device) {
        MPN_TRY(c->activity.ensure(bytes));
        out = (int32_t *)c->activity.p;
    }
    MPN_TRY(launch_activity(c->grid(), c->dist_bits, L, out, c->stream));
    if (!on_device)
        MPN_TRY(cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, c->stream));
    return from_cuda(cudaStreamSynchronize(c->stream));
}

static mpn_status trace_prepare(mpn_ctx *c, const uint32_t *starts, int32_t n,
                                const uint32_t **ds, uint64_t *total, bool euclid = false,
                                uint32_t *walk_max = nullptr) {
    if (!c || n < 0 || (n > 0 && !starts)) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    if (st != MPN_OK) return st;
    if (!c->propagated) return MPN_ESTATE;
    if (n > 0 && !is_device_ptr(starts)) {
        const uint64_t N = (uint64_t)c->H * c->W;
        for (int32_t i = 0; i < n; ++i)
            if ((uint64_t)starts[i] >= N) return MPN_EINVAL;
    }
    st = stage_u32(c, c->starts, starts, n, ds);
    if (st != MPN_OK) return st;
    MPN_TRY(c->offsets.ensure((size_t)(n + 1) * sizeof(uint64_t)));
    MPN_TRY(c->status.ensure((size_t)(n > 0 ? n : 1)));
    Ctl *ctl = (Ctl *)c->ctl.p;
    MPN_TRY(cudaMemsetAsync(&ctl->err, 0, sizeof(uint32_t), c->stream));
    MPN_TRY(cudaMemsetAsync(&ctl->walk_max, 0, sizeof(uint32_t), c->stream));
    MPN_TRY(cudaMemsetAsync(c->offsets.p, 0, sizeof(uint64_t), c->stream));
    if (n > 0) {
        MPN_TRY(launch_trace_lengths(c->grid(), c->dist_bits, *ds, n, (uint64_t *)c->offsets.p,
                                     (int8_t *)c->status.p, ctl, c->stream));
        if (euclid)   // straightened lengths replace d + 1
            MPN_TRY(launch_euclid(c->grid(), c->dist_bits, *ds, n, (uint64_t *)c->offsets.p,
                                  (const int8_t *)c->status.p, nullptr, false, c->stream, &ctl->err));
        MPN_TRY(launch_scan((uint64_t *)c->offsets.p, n, c->stream));
    }
    uint32_t err = 0;
    MPN_TRY(to_mbox(c, kMboxTotal, (uint64_t *)c->offsets.p + n, sizeof(uint64_t)));
    MPN_TRY(to_mbox(c, kMboxErr, &ctl->err, sizeof(uint32_t)));
    MPN_TRY(to_mbox(c, kMboxWalk, &ctl->walk_max, sizeof(uint32_t)));
    MPN_TRY(cudaStreamSynchronize(c->stream));
    memcpy(total, c->mbox + kMboxTotal, sizeof(uint64_t));
    memcpy(&err, c->mbox + kMboxErr, sizeof(uint32_t));
    if (walk_max) memcpy(walk_max, c->mbox + kMboxWalk, sizeof(uint32_t));
    if (err) return from_err_bits(err);
    return MPN_OK;
}

mpn_status mpn_trace_lengths(mpn_ctx *c, const uint32_t *starts, int32_t n, uint64_t *offsets) {
    if (!offsets) return MPN_EINVAL;
    const uint32_t *ds = nullptr;
    uint64_t total = 0;
    mpn_status st = trace_prepare(c, starts, n, &ds, &total);
    if (st != MPN_OK) return st;
    MPN_TRY(copy_out(c, offsets, c->offsets.p, (size_t)(n + 1) * sizeof(uint64_t)));
    return from_cuda(cudaStreamSynchronize(c->stream));
}

static mpn_status trace_any(mpn_ctx *c, const uint32_t *starts, int32_t n, uint64_t *offsets,
                            uint32_t *cells, uint64_t cells_cap, int8_t *status, bool euclid) {
    NvtxRange nvtx_range("mpn_trace");
    if (!offsets || (n > 0 && !status)) return MPN_EINVAL;
    const uint32_t *ds = nullptr;
    uint64_t total = 0;
    uint32_t walk_max = 0;
    mpn_status st = trace_prepare(c, starts, n, &ds, &total, euclid, &walk_max);
    if (st != MPN_OK) return st;
    MPN_TRY(copy_out(c, offsets, c->offsets.p, (size_t)(n + 1) * sizeof(uint64_t)));
    if (n > 0) MPN_TRY(copy_out(c, status, c->status.p, (size_t)n));
    if (total > cells_cap) {
        MPN_TRY(cudaStreamSynchronize(c->stream));
        return MPN_ENOMEM;
    }
    if (total > 0 && !cells) return MPN_EINVAL;
    const bool cells_dev = total > 0 && is_device_ptr(cells);
    uint32_t *dcells = cells;
    if (total > 0 && !cells_dev) {
        MPN_TRY(c->cells.ensure((size_t)total * sizeof(uint32_t)));
        dcells = (uint32_t *)c->cells.p;
    }
    Ctl *ctl = (Ctl *)c->ctl.p;
    MPN_TRY(cudaEventRecord(c->ev[4], c->stream));
    if (euclid)
        MPN_TRY(launch_euclid(c->grid(), c->dist_bits, ds, n, (uint64_t *)c->offsets.p,
                              (const int8_t *)c->status.p, dcells, true, c->stream, &ctl->err));
    else {
        // scratch for the longest-first walk order (no order if it cannot be had)
        uint32_t *ord = nullptr;
        if (c->order.ensure((size_t)n * sizeof(uint32_t)) == cudaSuccess) ord = (uint32_t *)c->order.p;
        else cudaGetLastError();
        // a walk far longer than the rest is split into segments walked side
        // by side (a jump table finds their first cells), when there is room
        bool split = false;
        const uint64_t seg_cap = total / kSegLen + (uint64_t)n + 1;
        if (walk_max > kLongWalk && seg_cap < 0xffffffffull) {
            const size_t cells_n = (size_t)c->H * c->W;
            if (c->jump.ensure(2 * cells_n * sizeof(uint32_t)) == cudaSuccess &&
                c->segs.ensure(seg_cap * sizeof(WalkSeg) + 16) == cudaSuccess)
                split = true;
            else
                cudaGetLastError();
        }
        if (split)
            MPN_TRY(launch_trace_split(c->grid(), c->dist_bits, ds, n, (const uint64_t *)c->offsets.p,
                                       (const int8_t *)c->status.p, dcells, ord, (uint32_t *)c->jump.p,
                                       (WalkSeg *)c->segs.p, (uint32_t)seg_cap,
                                       (uint32_t *)((char *)c->segs.p + seg_cap * sizeof(WalkSeg)),
                                       c->stream, &ctl->err));
        else
            MPN_TRY(launch_trace(c->grid(), c->dist_bits, ds, n, (const uint64_t *)c->offsets.p,
                                 (const int8_t *)c->status.p, dcells, ord, c->stream, &ctl->err));
    }
    MPN_TRY(cudaEventRecord(c->ev[5], c->stream));
    c->ev_trace = true;
    if (total > 0 && !cells_dev) MPN_TRY(copy_out(c, cells, dcells, (size_t)total * sizeof(uint32_t)));
    uint32_t err = 0;
    MPN_TRY(to_mbox(c, kMboxErr, &ctl->err, sizeof(uint32_t)));
    MPN_TRY(cudaStreamSynchronize(c->stream));
    memcpy(&err, c->mbox + kMboxErr, sizeof(uint32_t));
    if (err) return (err & ERR_TRACE) ? MPN_ECUDA : from_err_bits(err);
    return MPN_OK;
}

mpn_status mpn_trace(mpn_ctx *c, const uint32_t *starts, int32_t n, uint64_t *offsets,
                     uint32_t *cells, uint64_t cells_cap, int8_t *status) {
    return trace_any(c, starts, n, offsets, cells, cells_cap, status, false);
}

mpn_status mpn_trace_euclid(mpn_ctx *c, const uint32_t *starts, int32_t n, uint64_t *offsets,
                            uint32_t *cells, uint64_t cells_cap, int8_t *status) {
    return trace_any(c, starts, n, offsets, cells, cells_cap, status, true);
}

mpn_status mpn_nearest_targets(mpn_ctx *c, const uint32_t *starts, int32_t n, uint32_t *target,
                               uint32_t *dist) {
    if (!target) return MPN_EINVAL;
    const uint32_t *ds = nullptr;
    uint64_t total = 0;
    mpn_status st = trace_prepare(c, starts, n, &ds, &total);
    if (st != MPN_OK || n == 0) return st;
    const bool t_dev = is_device_ptr(target), d_dev = dist && is_device_ptr(dist);
    uint32_t *dt = target, *dd = dist;
    if (!t_dev || (dist && !d_dev)) {
        MPN_TRY(c->cells.ensure((size_t)n * 8));
        if (!t_dev) dt = (uint32_t *)c->cells.p;
        if (dist && !d_dev) dd = (uint32_t *)c->cells.p + n;
    }
    Ctl *ctl = (Ctl *)c->ctl.p;
    MPN_TRY(cudaEventRecord(c->ev[4], c->stream));
    MPN_TRY(launch_nearest(c->grid(), c->dist_bits, ds, n, (const int8_t *)c->status.p, dt, dd,
                           c->stream, &ctl->err));
    MPN_TRY(cudaEventRecord(c->ev[5], c->stream));
    c->ev_trace = true;
    if (!t_dev) MPN_TRY(copy_out(c, target, dt, (size_t)n * 4));
    if (dist && !d_dev) MPN_TRY(copy_out(c, dist, dd, (size_t)n * 4));
    uint32_t err = 0;
    MPN_TRY(to_mbox(c, kMboxErr, &ctl->err, sizeof(uint32_t)));
    MPN_TRY(cudaStreamSynchronize(c->stream));
    memcpy(&err, c->mbox + kMboxErr, sizeof(uint32_t));
    if (err) return (err & ERR_TRACE) ? MPN_ECUDA : from_err_bits(err);
    return MPN_OK;
}

mpn_status mpn_tune_query(int32_t H, int32_t W, int32_t variant, int32_t *depth, float *ms) {
    if (H < 1 || W < 1 || variant < 0 || variant >= num_variants()) return MPN_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune.mu);
    const int b = bucket_of(H, W);
    if (!g_tune.depth[b][variant]) return MPN_ESTATE;
    if (depth) *depth = g_tune.depth[b][variant];
    if (ms) *ms = g_tune.ms[b][variant];
    return MPN_OK;
}

mpn_status mpn_autotune(mpn_ctx *c, const uint32_t *targets, int32_t n, int32_t *variant,
                        int32_t *depth, float *best_ms) {
    NvtxRange nvtx_range("mpn_autotune");
    if (!c || !targets || n < 1) return MPN_EINVAL;
    static const int kDepths[] = {8, 12, 16, 20, 24, 28, 32};
    int bv = -1, bd = 0;
    float bms = 0.f;
    for (int v = 0; v < num_variants(); ++v) {
        for (int d : kDepths) {
            if (configure(c, v, d) != MPN_OK) continue;
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {   // the first run warms caches and clocks
                uint32_t layers = 0;
                mpn_status st = mpn_propagate(c, targets, n, 0, &layers);
                if (st != MPN_OK) return st;
                MPN_TRY(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
            }
            mpn::tune_record(c->H, c->W, v, d, ms);
            if (bv < 0 || ms < bms) {
                bv = v;
                bd = d;
                bms = ms;
            }
        }
    }
    if (bv < 0) return MPN_ECUDA;
    mpn_status st = configure(c, bv, bd);
    if (st != MPN_OK) return st;
    c->auto_tune = false;
    c->propagated = false;
    if (variant) *variant = bv;
    if (depth) *depth = bd;
    if (best_ms) *best_ms = bms;
    return MPN_OK;
}

mpn_status mpn_get_stats(mpn_ctx *c, mpn_stats *out) {
    if (!c || !out) return MPN_EINVAL;
    mpn_status st = finish_propagate(c);
    MPN_TRY(cudaStreamSynchronize(c->stream));
    std::memset(out, 0, sizeof(*out));
    out->H = c->H;
    out->W = c->W;
    out->pitch_words = c->P;
    out->dist_bits = c->dist_bits;
    out->variant = c->variant;
    out->depth = c->depth;
    out->tiles_x = c->ntx;
    out->tiles_y = c->nty;
    out->blocks = c->blocks;
    out->layers = c->last_layers;
    out->sweeps = c->last_ctl.sweeps;
    out->tile_visits = c->last_ctl.visits;
    out->tile_layers = c->last_ctl.tile_layers;
    out->log_entries = c->last_ctl.log_entries;
    // timings are best effort: a failed query leaves the last value and no
    // stale error behind for the next launch check
    if (c->ev_enc && cudaEventElapsedTime(&c->ms_encode, c->ev[0], c->ev[1]) != cudaSuccess)
        cudaGetLastError();
    if (c->ev_prop && cudaEventElapsedTime(&c->ms_propagate, c->ev[2], c->ev[3]) != cudaSuccess)
        cudaGetLastError();
    if (c->ev_trace && cudaEventElapsedTime(&c->ms_trace, c->ev[4], c->ev[5]) != cudaSuccess)
        cudaGetLastError();
    out->ms_encode = c->ms_encode;
    out->ms_propagate = c->ms_propagate;
    out->ms_trace = c->ms_trace;
    return st;
}

void mpn_destroy(mpn_ctx *c) {
    if (!c) return;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) cudaGetLastError();
    if (c->out_pending && cudaEventSynchronize(c->ev_out) != cudaSuccess) cudaGetLastError();
    DevBuf *bufs[] = {&c->free_bits, &c->state, &c->log, &c->dist, &c->ctl, &c->tiles,
                      &c->mask_stage, &c->targets, &c->starts, &c->offsets, &c->status,
                      &c->cells, &c->activity, &c->order, &c->jump, &c->segs, &c->check};
    for (DevBuf *b : bufs) b->release();
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->ev_ready) cudaEventDestroy(c->ev_ready);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->mbox) cudaFreeHost(c->mbox);
    delete c;
}

}  // extern "C"
