// Internal definitions shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "mpn.h"

namespace mpn {

// An NVTX range over a host-side library call (visible to profilers that
// record NVTX; a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// error bits the GPU records in Ctl::err
constexpr uint32_t ERR_TIMEOUT = 1u;    // a grid-wide wait hit its iteration limit
constexpr uint32_t ERR_OVERFLOW = 2u;   // a distance above 65534 in a uint16 plane
constexpr uint32_t ERR_INVAL = 4u;      // a target index out of range
constexpr uint32_t ERR_OBSTACLE = 8u;   // a target on an obstacle
constexpr uint32_t ERR_SWEEPS = 16u;    // sweep count past the provable bound
constexpr uint32_t ERR_TRACE = 32u;     // a walk found no neighbour one step closer

// Border zones of a tile interior touched by frontier cells (frontier = cells
// whose distance equals the last layer of a sweep). A zone bit says which
// tile (itself or one of its 8 neighbours) the frontier can reach within the
// next k layers, so that tile is queued for the next sweep.
constexpr uint32_t FB_ANY = 1u, FB_N = 2u, FB_S = 4u, FB_W = 8u, FB_E = 16u;
constexpr uint32_t FB_NW = 32u, FB_NE = 64u, FB_SW = 128u, FB_SE = 256u;

// Device control block of one propagation (zeroed before each run).
struct Ctl {
    unsigned int bar_count;        // grid-barrier arrivals of this launch (monotonic)
    unsigned int log_next;         // next free chunk of the activation log
    unsigned int work[4];          // claim counters of the tile lists, by sweep mod kListSlots
    unsigned int list_len[4];      // lengths of the tile lists, by sweep mod kListSlots
    unsigned int err;
    unsigned int max_layer;        // largest activation layer seen
    unsigned int sweeps;
    unsigned int plain_last;       // per-layer kernel: last layer that activated a cell
    unsigned int walk_max;         // longest path (cells) of the last trace's starts, saturated
    unsigned long long visits;     // tile visits
    unsigned long long tile_layers;   // layers those visits ran (a stable region stops early)
    unsigned long long log_entries;   // activation-log entries written
};

// Bit planes and distance plane of one grid. Bit b of word w in row y is cell
// x = 32 * w + b; rows are P words apart (P a multiple of 4).
//
// The propagation state keeps four words per plane word o, at state[4 * o]:
// {V, N0, V, N1}. V = reached; Np = the cells that the last sweep of parity p
// to change the word reached in it (0 after a sweep of the other parity
// changed it). Each {V, Np} pair is stored and loaded as one 64-bit access, so
// a reader always gets a word's reached bits together with the matching
// this-sweep bits, and neither side needs a fence.
struct GridDev {
    const uint32_t *free_bits;   // 1 = free; bits at x >= W are 0
    uint32_t *state;             // 4 * H * P words, see above
    void *dist;                  // H*W uint16 or uint32, row-major, pitch W
    int H, W, P;
};

// Tile queue of one propagation. Sweep s takes its tiles from list s mod
// kListSlots; an entry holds 1 + the tile id (0: not written yet), and the
// block that takes an entry clears it, so a list slot is all zeros again when
// it is reused. A tile is queued for sweep s at most once: stamps[s mod
// kStampSlots][t] = s + 1 once it is (only grows). done[t] = 1 + the last sweep
// whose visit of t has finished (its writes published). Visits of sweep s
// queue tiles for s + 1, and a block waiting at the end of sweep s may already
// run tiles of sweep s + 1 (which queue for s + 2), so three stamp arrays and
// four list slots keep every sweep's bookkeeping apart.
constexpr int kStampSlots = 3;
constexpr int kListSlots = 4;
// words per tile of the queue buffer before the visit slots: stamps, done,
// latest log header, logged-visit count, lists
constexpr int kTileQueueWords = kStampSlots + 1 + 2 + kListSlots;

// Counters behind the block ranks of a persistent launch (wave::block_rank):
// 256 per-SM counters, 32 per-place counters and a barrier counter.
constexpr uint32_t kRankWords = 320;

struct PropParams {
    GridDev g;
    uint32_t *stamps;            // kStampSlots arrays of ntiles: 1 + sweep the tile is queued for
    uint32_t *done;              // per tile: 1 + last sweep whose visit of it finished
    uint32_t *tile_head;         // per tile: 1 + log index of its latest visit header, 0 = none
    uint32_t *tile_nv;           // per tile: visits that logged entries
    uint4 *tile_vis;             // per tile: kTileSlots slots {header index, entry count, l0 + 1, 0} of visit n
    uint32_t *lists;             // kListSlots tile lists of ntx * nty entries (1 + tile id)
    Ctl *ctl;
    int ntx, nty;                // tiles
    int k;                       // temporal depth (layers per sweep), halo rows
    int TY;                      // interior rows per tile
    int TXW;                     // interior words per tile
    uint32_t max_layers;         // 0 = until nothing changes; else the last layer (absolute)
    uint32_t l_base;             // layer the run starts from: sweep s covers l_base + s k + 1 ..
    uint32_t spin_limit;         // barrier wait limit (iterations of ~100 ns)
    uint32_t lookahead;          // 1: blocks waiting at a sweep's end run ready tiles of the next
    uint32_t sweep_cap;          // more sweeps than this is an error
    uint32_t *log;               // activation log (log_chunks chunks), or null
    uint32_t log_chunks;
    uint32_t *rank;              // kRankWords counters, zero at the launch (block ranks), or null
};

// Activation log: instead of writing distances during a tile visit, the visit
// records, for every word of its interior in which it reached cells, one
// 32-byte entry of kLogFields words -- the word's place in the tile interior
// (row * TXW + word), the reached bits and the five Gray-code counter planes
// -- behind a header entry of the visit {1 + index of the tile's previous
// header (0 = none), entry count, layer of offset 0 (l0 + 1), the visit's
// number n among the tile's logged visits}. The header becomes the tile's
// latest (PropParams::tile_head, a chain through the headers), and for n <
// kTileSlots its index, count and layer also go to the tile's slot n. After
// the propagation k_log_decode gathers each tile's visits (the slots in
// parallel, later visits along the chain)
// and writes every cell of the tile's interior once, so the distance plane
// needs no fill beforehand. Entries are
// numbered globally; chunk c holds entries [c * kLogChunk, (c + 1) *
// kLogChunk), and a visit's header and entries lie in one chunk. Each block
// fills chunks it takes from a shared pool; a block that finds the pool
// empty writes its distances directly (and the decode keeps the cells it
// cannot account for: reached, with no entry).
constexpr uint32_t kLogChunk = 4096;
constexpr uint32_t kTileSlots = 64;
constexpr uint32_t kLogFields = 8;

// Words of the tile-queue buffer for ntiles tiles: the block-rank counters
// (kRankWords), kTileQueueWords per tile
// (stamps, done, latest header, logged-visit count, lists), then, 16-byte
// aligned, kTileSlots visit slots of 4 words per tile when with_slots.
inline size_t tile_queue_words(size_t ntiles, bool with_slots) {
    const size_t head = (kRankWords + kTileQueueWords * ntiles + 3) & ~(size_t)3;
    return head + (with_slots ? 4 * (size_t)kTileSlots * ntiles : 0);
}

// Point p's queue arrays into buf (tile_queue_words(ntiles, with_slots)
// words, 16-byte aligned): the block-rank counters, then the per-tile arrays.
// The first kRankWords + kTileQueueWords * ntiles words must be zero before
// each propagation (returned in *clear_words).
inline void layout_tile_queue(uint32_t *buf, size_t ntiles, bool with_slots, PropParams *p,
                              size_t *clear_words) {
    p->rank = buf;
    p->stamps = buf + kRankWords;
    p->done = p->stamps + kStampSlots * ntiles;
    p->tile_head = p->done + ntiles;
    p->tile_nv = p->tile_head + ntiles;
    p->lists = p->tile_nv + ntiles;
    p->tile_vis = with_slots
                      ? reinterpret_cast<uint4 *>(buf + ((kRankWords + kTileQueueWords * ntiles + 3) & ~(size_t)3))
                      : nullptr;
    *clear_words = kRankWords + kTileQueueWords * ntiles;
}

struct VariantDesc {
    int rxw;      // region words (lanes per row group x words per lane)
    int r;        // rows per lane
    int nwarps;   // warps per block that run the layers
    int minb;     // blocks per SM the register budget aims at
    int tma;      // 1: one more (producer) warp stages regions with TMA; uint32 planes only
    int wpl = 1;  // adjacent words of a row per lane
};

// Rows of a variant's region: warps x row groups per warp x rows per lane.
inline int region_rows(const VariantDesc &d) { return d.nwarps * (32 / (d.rxw / d.wpl)) * d.r; }

// ---- autotuner table (api.cu): best depth per (size bucket, variant) ----
// bucket = ceil(log2(max(H, W))); returns false when nothing was measured.
bool tune_lookup(int H, int W, int variant, int *depth);
bool tune_best(int H, int W, int *variant, int *depth);

// ---- launch helpers implemented in the .cu files ----
void count_launch(int n = 1);
// remember the last CUDA error a library call hit (per host thread), for
// mpn_last_error
void note_cuda_error(cudaError_t e);

int num_variants();
VariantDesc variant_desc(int v);
int variant_threads(int v);   // threads per block of variant v
cudaError_t propagate_blocks_per_sm(int v, int dist_bits, int *out);
cudaError_t launch_propagate(int v, int dist_bits, const PropParams &p, int blocks,
                             cudaStream_t st);
// k_log_decode over the whole plane (after k_propagate with a log); no-op
// without one. slots (1..kTileSlots, else kTileSlots): how many of a tile's
// visits the decode takes from its slots before the header chain.
cudaError_t launch_log_decode(const PropParams &p, int dist_bits, int sm_count, uint32_t slots,
                              cudaStream_t st);
cudaError_t launch_seed(const uint32_t *targets, int n, const PropParams &p, int dist_bits,
                        cudaStream_t st);
// Seed a run that resumes from a distance plane: cells at distance <= from
// (= p.l_base) are reached and keep their distance, all others start
// unreached; tiles with cells at distance `from` are queued for sweep 0. din
// (H * W of the dtype, device) may be the context's own plane.
cudaError_t launch_seed_plane(const void *din, const PropParams &p, int dist_bits, cudaStream_t st);
cudaError_t launch_plain_layer(const GridDev &g, int dist_bits, uint32_t layer, Ctl *ctl,
                               cudaStream_t st);
cudaError_t launch_plain_seed(const uint32_t *targets, int n, const GridDev &g, int dist_bits,
                              Ctl *ctl, cudaStream_t st);

cudaError_t launch_pack(const uint8_t *mask, int H, int W, int P, uint32_t *free_bits,
                        cudaStream_t st);
// launch_pack through a flat bit stream in `scratch` (at least H * W / 32 + 1
// words; clobbered): vector loads, for a 16-byte-aligned mask (otherwise it is
// launch_pack).
cudaError_t launch_pack_fast(const uint8_t *mask, int H, int W, int P, uint32_t *free_bits,
                             uint32_t *scratch, size_t scratch_words, cudaStream_t st);
cudaError_t launch_repack(const uint32_t *src, int H, int W, int src_pitch, int P,
                          uint32_t *free_bits, cudaStream_t st);

cudaError_t launch_trace_lengths(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                                 uint64_t *lens_or_offsets, int8_t *status, Ctl *ctl,
                                 cudaStream_t st);
cudaError_t launch_scan(uint64_t *offsets, int n, cudaStream_t st);
// order: n words of scratch for the longest-first walk order (uint32 planes),
// or null for the starts' own order
cudaError_t launch_trace(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                         const uint64_t *offsets, const int8_t *status, uint32_t *cells,
                         uint32_t *order, cudaStream_t st, uint32_t *err);
// Walks longer than kLongWalk cells are cut into segments of kSegLen steps,
// walked side by side: the cell kSegLen steps further along every walk comes
// from a jump table succ^kSegLen (succ = the next cell of the walk rule),
// built by repeated squaring in `jump` (2 * H * W words of scratch). segs:
// room for seg_cap segments (16 bytes each) and a counter at nseg.
constexpr uint32_t kLongWalk = 8192;
constexpr uint32_t kSegLen = 2048;
struct WalkSeg {
    uint32_t cell;    // first cell of the segment
    uint32_t dstop;   // distance at which it ends (its last cell)
    uint64_t out;     // where its first cell goes in the path output
};
cudaError_t launch_trace_split(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                               const uint64_t *offsets, const int8_t *status, uint32_t *cells,
                               uint32_t *order, uint32_t *jump, WalkSeg *segs, uint32_t seg_cap,
                               uint32_t *nseg, cudaStream_t st, uint32_t *err);
cudaError_t launch_activity(const GridDev &g, int dist_bits, uint32_t L, int32_t *out,
                            cudaStream_t st);
// Count the cells of the plane that break the distance-map invariants
// (mpn_check) into *count (device).
cudaError_t launch_check_plane(const GridDev &g, int dist_bits, uint32_t max_layers,
                               unsigned long long *count, cudaStream_t st);

// One grid of a batched trace: the paths of many grids are measured, ordered
// and walked together (a walk takes as long as its path, so the grids' walks
// run side by side in one launch, longest first across all of them).
struct WalkJob {
    GridDev g;                  // free_bits (for the start status), dist, H, W, P
    const uint32_t *starts;     // ns start cells
    uint64_t *offsets;          // ns + 1: path offsets (written by the lengths step)
    int8_t *status;             // ns: per-start status
    uint32_t *cells;            // path cells, or null: the walks of this grid are skipped
    int dist_bits;
    uint32_t ns;
    uint32_t walk_base;         // index of this grid's first walk among all walks of the batch
    uint32_t split;             // 1: its walks longer than kLongWalk go in segments (not here)
};
// Per job: status and path length of every start, offsets (scan), the job's
// path-cell total in totals[j] and its longest walk in totals[njobs + j], and
// every walk's length (saturated to 32 bits) in walk_len[walk_base + i].
cudaError_t launch_batch_lengths(const WalkJob *jobs, int njobs, uint32_t *walk_len,
                                 uint64_t *totals, uint32_t *err, cudaStream_t st);
// The walks of every job with cells, longest first (order: nwalks words of
// scratch).
cudaError_t launch_batch_walks(const WalkJob *jobs, int njobs, const uint32_t *walk_len,
                               uint32_t nwalks, uint32_t *order, uint32_t *err, cudaStream_t st);
// A segment of a long walk of batch job `job`.
struct BatchSeg {
    uint32_t cell, dstop, job, pad;
    uint64_t out;
};
// The jump table succ^kSegLen of one grid in `jump` (2 * H * W words);
// returns the half that holds it.
cudaError_t launch_jump_table(const GridDev &g, int dist_bits, uint32_t *jump, uint32_t **table,
                              cudaStream_t st);
// Segments of the walks of job j (on the device) longer than kLongWalk, added
// to segs (counter at nseg; room for cap).
cudaError_t launch_batch_segments(const WalkJob *jobs, int j, uint32_t ns, int dist_bits,
                                  const uint32_t *table, BatchSeg *segs, uint32_t cap, uint32_t *nseg,
                                  uint32_t *err, cudaStream_t st);
// Walk every segment (warp per segment; up to cap).
cudaError_t launch_batch_segwalks(const WalkJob *jobs, const BatchSeg *segs, const uint32_t *nseg,
                                  uint32_t cap, uint32_t *err, cudaStream_t st);
cudaError_t launch_nearest(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                           const int8_t *status, uint32_t *ends, uint32_t *ends_d, cudaStream_t st,
                           uint32_t *err);
cudaError_t launch_euclid(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                          uint64_t *offsets, const int8_t *status, uint32_t *cells, bool write,
                          cudaStream_t st, uint32_t *err);

}  // namespace mpn
