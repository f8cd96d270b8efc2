/*
 * mpn -- max-pooling path planner on GB300 (sm_103a). C ABI.
 *
 * The method (arXiv 2004.00540, "Generation of Paths in a Maze using a Deep
 * Network without Learning"): a stack of identical layers, each a 3x3
 * stride-1 max pool followed by adding the environment map I_e (0 free,
 * -maxint obstacle) and the source map I_s, then a ReLU (Methods, "Activity
 * Map Generation", Fig. 1). Activity spreads one cell per layer from the
 * sources; the layer at which a free cell first turns positive is its
 * 8-connected unit-cost hop distance d to the nearest source, and the final
 * activity map is O = L + 1 - d on reached cells. A path is read back from any
 * start by stepping to the neighbour with the largest activity, i.e. distance
 * d - 1 (Methods, "Path Reconstruction").
 *
 * Vocabulary: the paper calls the cells where activity starts "sources"; this
 * API calls them TARGETS (the cells paths lead to). Paths are traced from
 * STARTS. Cells are addressed by linear index y * W + x (row-major).
 *
 * Conventions for every call:
 *  - Every call returns an mpn_status; nothing aborts or exits.
 *  - Pointer arguments documented "host or device" are classified with
 *    cudaPointerGetAttributes: device (and managed) memory is read in place,
 *    anything else is treated as host memory and copied. Path, offset,
 *    status and nearest-target results bound for page-locked host memory are
 *    stored there by a small kernel (not a copy engine, whose device-to-host
 *    transfers queue behind other streams' large downloads), so such
 *    buffers must be writable by the device (not registered read-only).
 *  - Work is ordered on the context's stream (mpn_create's stream, or
 *    mpn_set_stream). A context is not thread-safe; separate contexts are
 *    independent. The caller owns every buffer it passes; the context owns
 *    the resident mask, distance plane and scratch until mpn_destroy.
 *  - Calls that do not need a host-visible result return before the GPU work
 *    finishes. An error the GPU detects (layer cap, distance overflow, a wait
 *    that timed out) is reported by the next call that synchronises
 *    (mpn_sync, mpn_get_distances, mpn_trace*, mpn_get_stats, or
 *    mpn_propagate with a non-NULL layers_run).
 */
#ifndef MPN_H
#define MPN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpn_ctx mpn_ctx;

typedef enum {
    MPN_OK = 0,
    MPN_EINVAL = 1,     /* bad argument: sizes < 1, index out of range, no targets */
    MPN_ENOMEM = 2,     /* device allocation failed, or an output capacity too small */
    MPN_ECUDA = 3,      /* a CUDA runtime call failed */
    MPN_ETIMEOUT = 4,   /* a grid-wide wait ran past its iteration limit */
    MPN_EOVERFLOW = 5,  /* a distance does not fit the uint16 plane */
    MPN_EOBSTACLE = 6,  /* a target lies on an obstacle */
    MPN_ESTATE = 7,     /* call out of order (trace before propagate) */
    MPN_ECHECK = 8      /* the on-device invariant check found violations (mpn_check) */
} mpn_status;

/* distance plane element type */
#define MPN_DIST_AUTO 0   /* uint16 if H*W <= 65535, else uint32 */
#define MPN_DIST_U16 16
#define MPN_DIST_U32 32
/* unreached cells and obstacles hold the all-ones sentinel of the dtype */
#define MPN_UNREACHED16 0xFFFFu
#define MPN_UNREACHED32 0xFFFFFFFFu

/* per-start trace status */
#define MPN_PATH_OK 0
#define MPN_PATH_UNREACHABLE 1
#define MPN_PATH_ON_OBSTACLE 2

/*
 * Create a context for one H x W grid and encode its mask (Methods, "Input":
 * the environment map I_e). mask: H*W uint8, row-major, nonzero = obstacle,
 * host or device. dist_bits: MPN_DIST_AUTO / _U16 / _U32. stream: a
 * cudaStream_t (NULL = legacy default stream). Allocates all device memory
 * the grid needs (mask bits, visit bits, distance plane, tile flags).
 * H, W >= 1 and H*W < 2^32 - 1, else MPN_EINVAL.
 */
mpn_status mpn_create(const uint8_t *mask, int32_t H, int32_t W, int32_t dist_bits,
                      void *stream, mpn_ctx **out);

/*
 * Like mpn_create, from an already packed FREE-cell bit plane: H rows of
 * pitch_words uint32 words; bit b of word w in row y is cell x = 32*w + b,
 * 1 = free. pitch_words >= ceil(W/32); bits at x >= W are ignored. Host or
 * device. Same environment map I_e as mpn_create (Methods, "Input": 0 on free
 * cells, -maxint on obstacles), given one bit per cell.
 */
mpn_status mpn_create_packed(const uint32_t *free_bits, int32_t H, int32_t W,
                             int32_t pitch_words, int32_t dist_bits, void *stream,
                             mpn_ctx **out);

/* Re-encode a new H*W uint8 mask of the same size (host or device), keeping
 * all allocations (Methods, "Input": a new environment map I_e for the same
 * network). Invalidates earlier distances. */
mpn_status mpn_set_mask(mpn_ctx *ctx, const uint8_t *mask);

/* Bind later work to another stream (a cudaStream_t). No counterpart in the
 * paper (stream plumbing). */
mpn_status mpn_set_stream(mpn_ctx *ctx, void *stream);

/*
 * Propagate activity from the targets (Methods, "Activity Map Generation";
 * the paper's I_s holds 1 at each target) and write the distance plane.
 * targets: n_targets >= 1 linear indices (uint32), host or device;
 * duplicates allowed. A target out of range gives MPN_EINVAL, one on an
 * obstacle MPN_EOBSTACLE (the paper's formula would make it a dead source).
 * max_layers = 0 runs until a layer activates no new cell (Methods,
 * "Determining the number of layers L", read as "stop at the first layer that
 * adds nothing"); max_layers = L > 0 is the paper's fixed-depth network of L
 * layers: cells with d > L stay unreached. layers_run (host, may be NULL):
 * receives the largest finite distance; passing it makes the call wait for
 * the GPU and report its errors.
 */
mpn_status mpn_propagate(mpn_ctx *ctx, const uint32_t *targets, int32_t n_targets,
                         uint32_t max_layers, uint32_t *layers_run);

/*
 * Continue the wave from a given distance plane: one more batch of layers,
 * with the activity of the last one passed back to its start (Results,
 * "Limitations and Practical Considerations": i iterations of up to L_max
 * layers when L is larger; and the recursive mode of Appendix, Table I). The
 * map is given as distances, d = L + 1 - O (Methods, "Activity Map
 * Generation"). dist_in: H*W elements of the context's dtype,
 * host or device; a cell with distance <= from_layer is reached at that
 * distance (it must be free, else MPN_EINVAL from the GPU); every other cell
 * starts unreached, whatever dist_in holds there. Layers from_layer + 1 ..
 * max_layers run (max_layers = 0: until a layer adds nothing; else it must be
 * > from_layer), and the context's distance plane gets the result: the kept
 * cells, then every cell reached by those layers at its first layer.
 * layers_run (may be NULL): the largest distance reached by those layers, 0
 * if none; passing it makes the call wait and report errors. This is how a
 * grid split into row strips over several GPUs advances: each strip runs k
 * layers from the plane it and its neighbours agree on, then they exchange
 * k-row halos.
 */
mpn_status mpn_propagate_resume(mpn_ctx *ctx, const void *dist_in, uint32_t from_layer,
                                uint32_t max_layers, uint32_t *layers_run);

/*
 * Same result as mpn_propagate, computed the way the paper's recursive mode
 * runs (Appendix, Table I: one layer per iteration): one kernel launch per
 * layer over the whole distance plane, with the host reading a "did anything
 * change" flag every check_every layers (>= 1). Baseline only.
 */
mpn_status mpn_propagate_plain(mpn_ctx *ctx, const uint32_t *targets, int32_t n_targets,
                               uint32_t max_layers, int32_t check_every,
                               uint32_t *layers_run);

/* Copy the distance plane (H*W elements of the context's dtype, row-major)
 * to dst; dst_on_device selects cudaMemcpyDeviceToDevice vs DeviceToHost.
 * Waits for the copy. MPN_ESTATE before the first propagate. The plane holds
 * each cell's first-activation layer d, from which the paper's activity map
 * is O = L + 1 - d (Methods, "Activity Map Generation"; mpn_get_activity
 * returns O itself). */
mpn_status mpn_get_distances(mpn_ctx *ctx, void *dst, int32_t dst_on_device);

/*
 * Enqueue the same copy (dst: host or device, H*W elements of the context's
 * dtype) on `stream` (a cudaStream_t; NULL: the context's stream), ordered
 * after the context's work so far, and return without waiting for it. The
 * last propagate's errors are reported first (which waits for that propagate
 * if no call has collected them yet). dst must not be read or freed until the
 * stream has passed the copy: synchronize that stream, or call mpn_sync on
 * this context. A later propagate on this context waits, on the device, for
 * the copy before it rewrites the plane. MPN_ESTATE before the first
 * propagate. The paper has no counterpart: it lets a caller download one
 * solve's distances while the next solve's mask goes up and its kernels run.
 */
mpn_status mpn_get_distances_async(mpn_ctx *ctx, void *dst, void *stream);

/*
 * The paper's final activity map O after L layers (Methods, "Activity Map
 * Generation"): O = L + 1 - d where d <= L, 0 elsewhere (obstacles,
 * unreached, farther than L). dst: H*W int32, device or host
 * (dst_on_device). L = 0 means the layer count of the last propagate.
 */
mpn_status mpn_get_activity(mpn_ctx *ctx, uint32_t L, int32_t *dst, int32_t dst_on_device);

/*
 * Path lengths only (for sizing): offsets[0] = 0 and offsets[i+1] -
 * offsets[i] = d(start_i) + 1 cells for a reachable start, 0 otherwise
 * (Methods, "Path Reconstruction": a path from a start at distance d takes d
 * steps, one layer of activity per step). starts: n >= 0 uint32 linear
 * indices, host or device. offsets: n+1 uint64, host or device. Waits for the
 * GPU.
 */
mpn_status mpn_trace_lengths(mpn_ctx *ctx, const uint32_t *starts, int32_t n,
                             uint64_t *offsets);

/*
 * Simple path reconstruction (Methods, "Path Reconstruction") from every
 * start: start first, then repeatedly the 8-neighbour with distance d - 1 --
 * among several, the one with the lowest linear index (the paper picks at
 * random) -- until a target (d = 0). Output in CSR form, host or device
 * buffers:
 *   offsets[n+1] uint64, cells[offsets[n]] uint32, status[n] int8
 *   (MPN_PATH_OK / _UNREACHABLE / _ON_OBSTACLE; empty path unless OK).
 * If offsets[n] > cells_cap, offsets and status are still written and the
 * call returns MPN_ENOMEM so the caller can resize. A start index out of
 * range is MPN_EINVAL. MPN_ESTATE before the first propagate. Waits for the
 * GPU once (to size the output).
 */
mpn_status mpn_trace(mpn_ctx *ctx, const uint32_t *starts, int32_t n, uint64_t *offsets,
                     uint32_t *cells, uint64_t cells_cap, int8_t *status);

/*
 * Euclidean path reconstruction (Methods, "Path Reconstruction", Eq. 1 and
 * the straightening that follows it): from each start, step to the
 * 4-neighbour (left, right, up, down, in Eq. 1's order) with the largest
 * activity, i.e. distance d - 1; then drop every point whose neighbours on
 * the path are sqrt(2) apart. Eq. 1 does not say what happens when no
 * 4-neighbour is one step closer (the closer cell is diagonal); this library
 * steps to the first 4-neighbour at the same distance that is 4-adjacent to a
 * closer cell (the corner of the diagonal move), or, if both corners are
 * obstacles, takes the diagonal step. Straightening scans forward: P(t) is
 * dropped when the last kept point and P(t+1) are sqrt(2) apart. Output and
 * errors as in mpn_trace (offsets[i+1] - offsets[i] = straightened length).
 */
mpn_status mpn_trace_euclid(mpn_ctx *ctx, const uint32_t *starts, int32_t n, uint64_t *offsets,
                            uint32_t *cells, uint64_t cells_cap, int8_t *status);

/*
 * Nearest target of each start (the paper's multi-source, multi-target use:
 * each customer's closest taxi, Results, "Multi-source Multi-target Path
 * Planning"): the target that simple path reconstruction from the start ends
 * at -- one of the nearest targets, chosen by the lowest-index descent -- and
 * the start's distance to it, without storing the paths. target[n] and
 * dist[n] (dist may be NULL), uint32, host or device; 0xFFFFFFFF for a start
 * that is unreachable or on an obstacle. Errors as in mpn_trace.
 */
mpn_status mpn_nearest_targets(mpn_ctx *ctx, const uint32_t *starts, int32_t n,
                               uint32_t *target, uint32_t *dist);

/*
 * On-device check of the last propagation's distance plane against what a
 * multi-source, 8-connected, unit-cost distance map must satisfy (Methods,
 * "Activity Map Generation": a cell first activates one layer after its most
 * active neighbour): every reached cell other than a target has a neighbour at
 * distance d - 1; two reached neighbours differ by at most 1; a free
 * neighbour of a reached cell is reached, unless the fixed depth (max_layers)
 * stopped the wave there; obstacles are unreached. *violations (may be NULL):
 * cells that break one of these. Returns MPN_ECHECK if there are any, else
 * MPN_OK; waits for the GPU. MPN_ESTATE before the first propagate. With the
 * environment variable MPN_CHECK=1, every mpn_propagate that waits
 * (layers_run non-NULL) runs this check too and returns MPN_ECHECK on a
 * violation (a debug mode; it reads the whole plane once more).
 */
mpn_status mpn_check(mpn_ctx *ctx, uint64_t *violations);

/* Wait for the context's stream and for its pending asynchronous distance
 * copy (mpn_get_distances_async); report any error the GPU recorded. No
 * counterpart in the paper (stream plumbing). */
mpn_status mpn_sync(mpn_ctx *ctx);

/* Free every device and host resource of the context (NULL is a no-op). No
 * counterpart in the paper (resource plumbing). */
void mpn_destroy(mpn_ctx *ctx);

/* Name of a status code. No counterpart in the paper. */
const char *mpn_status_str(mpn_status s);

/*
 * Propagation tiling (no counterpart in the paper, which runs one library
 * max-pool per layer; here k layers of Methods, "Activity Map Generation", run
 * per tile visit). variant: index into the compiled tile shapes
 * (mpn_variant_info); depth: temporal blocking depth k = layers advanced per
 * tile visit, 1..32 (also the halo width in rows), with region_rows - 2k >= k
 * (the interior must be at least as tall as the halo), else MPN_EINVAL.
 * variant < 0 restores the automatic choice.
 */
mpn_status mpn_set_tuning(mpn_ctx *ctx, int32_t variant, int32_t depth);

/*
 * Autotuner (no counterpart in the paper; its run time depends on L and n,
 * Results, "Run-time"): time every compiled tile shape and every depth in {8, 12, 16,
 * 20, 24, 28, 32} (where the shape allows it) by propagating from these targets on
 * this context's grid; keep the fastest for the context and record, for the
 * grid's size bucket ceil(log2(max(H, W))), the fastest depth per shape and
 * the fastest shape overall. Contexts created later with automatic tiling,
 * and batches (for their shape), start from the recorded choice. Leaves the
 * context without distances (propagate again). Outputs may be NULL.
 */
mpn_status mpn_autotune(mpn_ctx *ctx, const uint32_t *targets, int32_t n_targets,
                        int32_t *variant, int32_t *depth, float *best_ms);

/* What the autotuner recorded for the size bucket of an H x W grid
 * (ceil(log2(max(H, W)))) and tile shape `variant`: the fastest depth and its
 * propagation time in ms (either output may be NULL). Batches use that depth
 * for grids of this bucket. MPN_ESTATE if nothing was measured for it,
 * MPN_EINVAL for sizes < 1 or an unknown shape. No counterpart in the paper. */
mpn_status mpn_tune_query(int32_t H, int32_t W, int32_t variant, int32_t *depth, float *ms);

/* Shape of compiled tile variant v: region rows, region words (32 cells
 * each), threads per block. MPN_EINVAL past the last variant. No counterpart
 * in the paper. */
mpn_status mpn_variant_info(int32_t v, int32_t *region_rows, int32_t *region_words,
                            int32_t *threads);

typedef struct {
    int32_t H, W, pitch_words, dist_bits;
    int32_t variant, depth;          /* tiling in use */
    int32_t tiles_x, tiles_y, blocks;
    uint32_t layers;                 /* largest finite distance of the last propagate */
    uint32_t sweeps;                 /* grid-wide rounds of the last propagate */
    uint64_t tile_visits;            /* tile visits of the last propagate */
    float ms_encode, ms_propagate, ms_trace;   /* device time of the last call of each */
    uint64_t tile_layers;            /* layers those tile visits ran: a visit stops early once
                                        its region is stable, so tile_layers / (tile_visits *
                                        depth) is the fraction of tile-layers executed */
    uint64_t log_entries;            /* activation-log entries (one per word and visit that
                                        reached cells in it) the last propagate wrote */
} mpn_stats;

/* Statistics of the last calls (waits for the GPU). layers is the paper's L,
 * the number of layers the network needs (Methods, "Determining the number of
 * layers L"); the rest has no counterpart in the paper. */
mpn_status mpn_get_stats(mpn_ctx *ctx, mpn_stats *out);

/* Number of kernels this library has launched in this process. No
 * counterpart in the paper (measurement). */
uint64_t mpn_launch_count(void);

/* Text of the last CUDA runtime error behind an MPN_ECUDA / MPN_ENOMEM
 * returned to this host thread ("" if none). No counterpart in the paper. */
const char *mpn_last_error(void);

/* ------------------------------------------------------------------------
 * Batched and continuously batched solving of many grids.
 *
 * A batch owns one device arena of budget_bytes and a table of grid slots.
 * mpn_batch_submit admits one grid (mask, targets, starts; host or device
 * pointers, copied into the arena) if its bit planes and results fit in the
 * arena now -- admission by device memory -- and returns MPN_ENOMEM
 * otherwise, so the caller can retry after other grids are released.
 * mpn_batch_run runs one round: grids submitted since the last round are
 * seeded, then one persistent launch advances every admitted grid (their
 * tiles share one work queue; each grid keeps its own layer clock) for up to
 * max_sweeps sweeps (0 = until all converge). Grids that converged are
 * traced at the end of the round (paths as in mpn_trace) and their bit planes
 * are freed; their distance plane and paths stay until mpn_batch_release.
 * (When a grid's paths do not fit in the arena at that moment, they are
 * traced when mpn_batch_result asks for them: straight into a device `cells`
 * buffer, or through a temporary device buffer for a host one -- the one
 * allocation outside the budget.)
 * Grids submitted while others are in flight join at the next round, so
 * their work overlaps on the device. A round (device-side preparation plus
 * the cooperative launch) is captured once per max_sweeps value as a CUDA
 * graph and replayed; its launch parameters never change because the
 * per-round state lives in device memory. Results are the same as one grid solved
 * alone with mpn_create/mpn_propagate/mpn_trace (bit for bit).
 *
 * The paper solves one map per network run and has no batch; each grid of a
 * batch goes through the same layers (Methods, "Activity Map Generation") and
 * the same simple path reconstruction (Methods, "Path Reconstruction"). The
 * batch calls below that only manage memory, tickets and rounds have no
 * counterpart in the paper.
 * ------------------------------------------------------------------------ */
typedef struct mpn_batch mpn_batch;

#define MPN_BATCH_PENDING 0
#define MPN_BATCH_DONE 1
#define MPN_BATCH_FAILED 2

typedef struct {
    uint64_t arena_bytes, arena_used, tiles_used;
    uint32_t next_sweep;        /* global sweep counter */
    uint64_t rounds, sweeps;    /* rounds run, sweeps run in total */
    float last_round_ms;        /* device time of the last round's propagation */
    int32_t blocks;             /* persistent blocks per launch */
    int32_t admitted, running, done, failed;
    int32_t graph;              /* 1: rounds replay a captured CUDA graph */
} mpn_batch_stats_t;

/* budget_bytes >= 1 MiB: the arena; variant: compiled tile shape 0, 1 or 12
 * (-1 = 0; other shapes are MPN_EINVAL); stream: cudaStream_t. */
mpn_status mpn_batch_create(uint64_t budget_bytes, int32_t variant, void *stream,
                            mpn_batch **out);

/* Temporal depth used for grids submitted from now on (1..32, 0 = default). */
mpn_status mpn_batch_set_depth(mpn_batch *b, int32_t depth);

/* Scheduling of a batch's rounds (no counterpart in the paper, which solves
 * one grid at a time). 1 (the default): every grid keeps its own sweep
 * clock; a grid's next sweep starts as soon as its own tiles of the current
 * one are done, and sweeps of at most 24 tiles are taken before larger ones,
 * so a grid that needs many sweeps of few tiles (a maze) does not wait for
 * the sweeps of large grids; a round's sweep budget counts each grid's own
 * sweeps. 0: all grids advance together, one sweep of every grid per sweep
 * of the launch (blocks waiting at a sweep's end run ready tiles of the
 * next). Results are the same bit for bit. Only while the batch holds no
 * grid (else MPN_ESTATE); shape 0, 1 or 12. */
mpn_status mpn_batch_set_mode(mpn_batch *b, int32_t per_grid_clock);

/* Admit one grid. dist_bits as in mpn_create; max_layers as in
 * mpn_propagate. *ticket identifies it. MPN_ENOMEM: it does not fit now.
 * End-points are checked here (the call waits for that): a target or start
 * out of range is MPN_EINVAL, a target on an obstacle MPN_EOBSTACLE, and the
 * grid is not admitted. A grid whose distances overflow a uint16 plane ends
 * FAILED (MPN_EOVERFLOW). */
mpn_status mpn_batch_submit(mpn_batch *b, const uint8_t *mask, int32_t H, int32_t W,
                            const uint32_t *targets, int32_t n_targets,
                            const uint32_t *starts, int32_t n_starts, int32_t dist_bits,
                            uint32_t max_layers, uint64_t *ticket);

/* One round (waits for it). max_sweeps: the round's sweep budget, 0 = until
 * every grid converged. With one clock for all grids a round runs at most
 * max_sweeps sweeps; with per-grid clocks every grid runs at least
 * max_sweeps of its own sweeps (or converges), and one whose sweeps are
 * faster runs on, up to 16 x max_sweeps, until every grid of the round has
 * run max_sweeps. n_running: grids admitted or in flight after the round;
 * n_done: grids finished (done or failed) and not yet released. */
mpn_status mpn_batch_run(mpn_batch *b, uint32_t max_sweeps, int32_t *n_running,
                         int32_t *n_done);

/* *state = MPN_BATCH_PENDING / _DONE / _FAILED (then returns its error). */
mpn_status mpn_batch_poll(mpn_batch *b, uint64_t ticket, int32_t *state);

/* Run rounds of max_sweeps sweeps (0: to convergence) until grid `ticket`
 * is DONE or FAILED; *state as in mpn_batch_poll (may be NULL). Other grids
 * advance with it. Returns the grid's status like mpn_batch_poll, an error of
 * a round, or MPN_ETIMEOUT after 2^20 rounds without an outcome. (The paper's
 * one-shot network has no batch; this is the blocking form of run + poll.) */
mpn_status mpn_batch_wait(mpn_batch *b, uint64_t ticket, uint32_t max_sweeps, int32_t *state);

/* Results of a DONE grid (any pointer may be NULL; host or device):
 * dist H*W of its dtype, offsets[n_starts+1], cells[offsets[n]] (MPN_ENOMEM if
 * cells_cap is smaller), status[n_starts], *layers. */
mpn_status mpn_batch_result(mpn_batch *b, uint64_t ticket, void *dist, uint64_t *offsets,
                            uint32_t *cells, uint64_t cells_cap, int8_t *status,
                            uint32_t *layers);

/* Shape, dtype and path-cell count of a submitted grid. */
mpn_status mpn_batch_info(mpn_batch *b, uint64_t ticket, int32_t *H, int32_t *W,
                          int32_t *dist_bits, uint64_t *total_cells);

/* Free a finished grid's arena space and slot. MPN_ESTATE while in flight. */
mpn_status mpn_batch_release(mpn_batch *b, uint64_t ticket);

mpn_status mpn_batch_stats(mpn_batch *b, mpn_batch_stats_t *out);

void mpn_batch_destroy(mpn_batch *b);

/*
 * Distances for one grid without allocating any memory. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory (code running inside another framework's memory pool or a
 * fixed-budget allocator, processes that must not grow after start-up,
 * real-time loops where an allocation and its implied synchronisation are not
 * allowed).
 *
 * Computes what mpn_create + mpn_propagate + mpn_get_distances compute for a
 * uint32 plane. All pointers are DEVICE memory owned by the caller:
 *   mask     H*W uint8, nonzero = obstacle;
 *   targets  n_targets >= 1 linear indices;
 *   dist     H*W uint32 output (0xFFFFFFFF = unreached or obstacle).
 * max_layers as in mpn_propagate. Work is ordered on `stream`; the call waits
 * for it to report errors (MPN_EINVAL for a target out of range,
 * MPN_EOBSTACLE for one on an obstacle).
 *
 * Limit: H <= 2048 and W <= 2048; larger grids return MPN_EINVAL, and so does
 * a mask, targets or dist pointer that is not memory of the current device.
 * The scratch (bit planes, tile queue, control block; about 2.6 MB) is one
 * fixed device array that every GPU on which this library's device code is
 * loaded holds until the process exits; with lazy module loading (the CUDA
 * default) that happens at the first use on the device, so the first call
 * there (or a warm-up call at start-up) is when the footprint grows. Calls
 * never call cudaMalloc/cudaFree or any allocating routine. The first call on
 * each device (and the first after a reset of it) looks up that array's device
 * address (cudaGetSymbolAddress) as its set-up, so make it before any stream
 * capture. Every call waits for its stream to finish (it reads the GPU's
 * error word back to the host) before it returns. All calls share the array
 * and each clears what must start at zero; calls whose GPU work overlaps
 * (other streams, other host threads) race on it.
 */
mpn_status mpn_propagate_noalloc(const uint8_t *mask, int32_t H, int32_t W,
                                 const uint32_t *targets, int32_t n_targets,
                                 uint32_t max_layers, uint32_t *dist, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPN_H */
