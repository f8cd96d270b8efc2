// Batched and continuously batched solving of many grids.
//
// A batch owns one device arena (its memory budget) and a table of grid slots.
// mpn_batch_submit admits a grid if its planes fit in the arena (admission by
// device memory) and gives it a range of global tile ids. mpn_batch_run runs
// one round: grids admitted since the last round are encoded and seeded, then
// ONE persistent launch advances every admitted grid -- tiles of all grids
// share one work queue -- for up to a given number of sweeps, or until every
// grid has converged. Each grid keeps its own layer clock (the sweep it
// started at), so grids submitted while others are in flight join at the
// next round and their work overlaps on the device. Grids that converge are
// traced at the end of the round, release their bit planes, and keep their
// distance plane and paths until mpn_batch_release.
//
// The per-tile work is wave::visit_tile, the same as the single-grid kernel.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "mpn_internal.cuh"
#include "wave.cuh"

namespace mpn {
namespace {

using wave::ld_acquire;
using wave::ld_relaxed;

// Device descriptor of one admitted grid.
struct MazeDesc {
    GridDev g;
    int dist_bits;
    int ntx, nty, TY, TXW, k;
    uint32_t tile_base;     // first global tile id
    uint32_t start_sweep;   // global sweep at which its layer 0 began
    uint32_t max_layers;    // 0 = until convergence
    uint32_t maxl;          // largest layer reached (atomicMax)
    uint32_t last_push;     // 1 + last sweep one of its tiles was queued for
    uint32_t err;           // ERR_* bits of this grid
    uint32_t pad;
    // per-grid sweep clock (the batch's per-grid mode)
    uint32_t ls;            // the grid's sweep in progress, or the next one to run
    uint32_t pend;          // visits of sweep ls not finished yet
    uint32_t cnt[2];        // tiles queued in its list slot q (sweep parity q)
    uint32_t ls0;           // ls when the round started
    uint32_t fstate;        // kFlowIdle / kFlowReady / kFlowRun / kFlowDone
};

constexpr uint32_t kFlowIdle = 0, kFlowReady = 1, kFlowRun = 2, kFlowDone = 3;
// a sweep of at most this many tiles goes to the priority ring (the 256-grid
// round: 4 tiles 158 ms, 8: 148, 16: 128, 24: 127, 32: 127, 64: 138, 256: 158)
constexpr uint32_t kFlowSmall = 24;

// A counter alone in its 128-byte line (the per-grid mode's counters are
// polled by idle blocks; sharing a line would slow every claim).
struct alignas(128) LineWord {
    uint32_t v;
    uint32_t pad[31];
};

struct BatchCtl {
    Ctl c;
    uint32_t next_sweep;    // global sweep the next round starts at
    uint32_t pad[3];
    // per-grid mode: two ticket rings (0: sweeps of few tiles, taken first)
    LineWord head[2];       // tickets claimed
    LineWord tail[2];       // tickets reserved by their publishers
    LineWord active;        // grids of the round neither converged nor paused
    LineWord reached;       // grids of the round that ran the sweep budget (or converged first)
    uint32_t round_grids;   // grids the round started with
    uint32_t pad3[31];
};

struct BatchParams {
    MazeDesc *descs;
    uint32_t *tile_maze;    // global tile id -> slot
    uint32_t *stamps;       // kStampSlots arrays of max_tiles: 1 + sweep the tile is queued for
    uint32_t *done;         // global tile id -> 1 + last sweep whose visit of it finished
    uint32_t *lists;        // kListSlots lists of max_tiles entries (1 + global tile id)
    uint32_t max_tiles;
    BatchCtl *bc;
    uint32_t round_sweeps;  // 0 = until every grid converged
    uint32_t spin_limit;
    uint32_t lookahead;     // 1: blocks waiting at a sweep's end run ready tiles of the next
    uint32_t *rank;         // kRankWords counters, zero at the launch (block ranks)
    uint32_t *ring;         // per-grid mode: 2 rings of ring_mask + 1 tickets (1 + global tile id)
    uint32_t ring_mask;
};

struct SeedJob {
    uint32_t slot;
    uint32_t n;
    const uint32_t *targets;
};

// Queue global tile gt of grid `slot` for sweep s unless it is queued already
// (the list entry holds 1 + gt, so a block waiting at the end of the previous
// sweep can poll it).
__device__ __forceinline__ void push_gt_b(const BatchParams &p, uint32_t slot, uint32_t gt, uint32_t s) {
    if (atomicMax(p.stamps + (size_t)(s % kStampSlots) * p.max_tiles + gt, s + 1) < s + 1) {
        const uint32_t sl = s % kListSlots;
        const uint32_t i = atomicAdd(&p.bc->c.list_len[sl], 1u);
        wave::st_relaxed(p.lists + (size_t)sl * p.max_tiles + i, gt + 1u);
        atomicMax(&p.descs[slot].last_push, s + 1);
    }
}

__device__ __forceinline__ void push_tile_b(const BatchParams &p, const MazeDesc &d, uint32_t slot,
                                            int ty, int tx, uint32_t s) {
    if (ty < 0 || tx < 0 || ty >= d.nty || tx >= d.ntx) return;
    push_gt_b(p, slot, d.tile_base + (uint32_t)(ty * d.ntx + tx), s);
}

// Take entry i of a tile list: the global tile id (-1 if never written), and
// clear the entry for the list slot's next use.
__device__ __forceinline__ int take_entry_b(uint32_t *list, uint32_t i) {
    const uint32_t e = ld_relaxed(list + i);
    if (e) wave::st_relaxed(list + i, 0u);
    return (int)e - 1;
}

// The tile of grid d that frontier cells in border zone z (one FB_* bit) of
// its tile (ty, tx) can reach, as a global tile id, or -1 past the grid's edge.
__device__ __forceinline__ int64_t zone_tile_b(const MazeDesc &d, int ty, int tx, uint32_t z) {
    if (z & (FB_N | FB_NW | FB_NE)) --ty;
    if (z & (FB_S | FB_SW | FB_SE)) ++ty;
    if (z & (FB_W | FB_NW | FB_SW)) --tx;
    if (z & (FB_E | FB_NE | FB_SE)) ++tx;
    if (ty < 0 || tx < 0 || ty >= d.nty || tx >= d.ntx) return -1;
    return (int64_t)d.tile_base + ty * d.ntx + tx;
}

__device__ void push_zone_b(const BatchParams &p, const MazeDesc &d, uint32_t slot, int ty, int tx,
                            uint32_t zone, uint32_t s) {
    if (zone & FB_ANY) push_tile_b(p, d, slot, ty, tx, s);
    if (zone & FB_N) push_tile_b(p, d, slot, ty - 1, tx, s);
    if (zone & FB_S) push_tile_b(p, d, slot, ty + 1, tx, s);
    if (zone & FB_W) push_tile_b(p, d, slot, ty, tx - 1, s);
    if (zone & FB_E) push_tile_b(p, d, slot, ty, tx + 1, s);
    if (zone & FB_NW) push_tile_b(p, d, slot, ty - 1, tx - 1, s);
    if (zone & FB_NE) push_tile_b(p, d, slot, ty - 1, tx + 1, s);
    if (zone & FB_SW) push_tile_b(p, d, slot, ty + 1, tx - 1, s);
    if (zone & FB_SE) push_tile_b(p, d, slot, ty + 1, tx + 1, s);
}

// Per-grid mode: queue global tile gt of grid `slot` for the grid's sweep s
// in the grid's own list slot s mod 2 (entries from tile_base on; a tile is
// queued at most once per sweep, so the grid's tile count bounds the list).
__device__ __forceinline__ void push_flow(const BatchParams &p, uint32_t slot, uint32_t gt, uint32_t s) {
    if (atomicMax(p.stamps + gt, s + 1u) < s + 1u) {
        MazeDesc &d = p.descs[slot];
        const uint32_t q = s & 1u;
        const uint32_t i = atomicAdd(&d.cnt[q], 1u);
        wave::st_relaxed(p.lists + (size_t)q * p.max_tiles + d.tile_base + i, gt + 1u);
    }
}

// One block per admitted grid: distance 0 and the reached bit at its
// targets, and its first tiles queued for the round's first sweep (per-grid
// mode: for the grid's own sweep 0).
__global__ void k_batch_seed(BatchParams p, const SeedJob *jobs, uint32_t flow) {
    const SeedJob job = jobs[blockIdx.x];
    const MazeDesc d = p.descs[job.slot];
    const uint32_t S = d.start_sweep;
    for (uint32_t i = threadIdx.x; i < job.n; i += blockDim.x) {
        const uint32_t t = job.targets[i];
        if ((uint64_t)t >= (uint64_t)d.g.H * (uint64_t)d.g.W) {
            atomicOr(&p.descs[job.slot].err, ERR_INVAL);
            continue;
        }
        const int y = (int)(t / (uint32_t)d.g.W), x = (int)(t % (uint32_t)d.g.W);
        const size_t wo = (size_t)y * d.g.P + (x >> 5);
        const uint32_t bit = 1u << (x & 31);
        if (!(d.g.free_bits[wo] & bit)) {
            atomicOr(&p.descs[job.slot].err, ERR_OBSTACLE);
            continue;
        }
        if (d.dist_bits == 16) reinterpret_cast<uint16_t *>(d.g.dist)[t] = 0;
        else reinterpret_cast<uint32_t *>(d.g.dist)[t] = 0u;
        atomicOr(d.g.state + 4 * wo, bit);   // V of both pairs
        atomicOr(d.g.state + 4 * wo + 2, bit);
        const int ty = y / d.TY, tx = (x >> 5) / d.TXW;
        const int ri = y - ty * d.TY, wi = (x >> 5) - tx * d.TXW;
        const uint32_t zone = wave::border_bits(ri, wi, bit, d.k, d.TY, d.TXW);
        if (!flow) {
            push_zone_b(p, d, job.slot, ty, tx, zone, S);
            continue;
        }
        for (int z = 0; z < 9; ++z) {
            if (!(zone & (1u << z))) continue;
            const int64_t gt = zone_tile_b(d, ty, tx, 1u << z);
            if (gt >= 0) push_flow(p, job.slot, (uint32_t)gt, 0u);
        }
    }
}

// The round's sweeps over every admitted grid's queued tiles. As in the
// single-grid kernel, entries 0 .. blocks - 1 of a sweep's list go one per
// block without an atomic, a visit's queue pushes are split across the next
// visit (stamp after the visit, append after the next visit's layers), and a
// block that has arrived at the end of a sweep runs tiles of the next sweep
// whose 3 x 3 neighbourhood (within their grid) has finished the sweep. A
// round's last sweep (the sweep budget) has no lookahead, so a round ends
// with every visit of its sweeps done and nothing run ahead.
template <int RXW, int R, int NW, int MINB, int WPL = 1>
__global__ void __launch_bounds__(NW * 32, MINB) k_batch_propagate(BatchParams p) {
    __shared__ wave::VisitSmem<RXW, NW, WPL> sm;
    __shared__ int s_tile;
    __shared__ unsigned s_mask[2], s_lastj[2], s_done;
    __shared__ uint32_t s_len;   // length of this sweep's list
    __shared__ int s_dec[2];     // end of sweep, by poll parity: -3 stop, -2 wait, -1 go on, >= 0 run tile
    __shared__ int s_done_t;     // visited tile whose done stamp is not out yet (-1: none)
    __shared__ uint32_t s_done_v;
    Ctl *ctl = &p.bc->c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned vq = 0u;
    unsigned long long blk_visits = 0;
    int pend_mine = -1;          // thread 0: list index claimed while waiting, not yet run
    const uint32_t s0 = ld_acquire(&p.bc->next_sweep);
    const uint32_t G = gridDim.x;
    const size_t MT = p.max_tiles;
    sm.zero_pad();   // (the first barrier below publishes it)
    int rk = 0;   // thread 0: this block's rank in the lists' fixed deal (wave::block_rank)
    if (threadIdx.x == 0) {
        rk = wave::block_rank(p.rank, p.spin_limit, &ctl->err);
        s_dec[0] = rk >= 0 ? 0 : -3;
        // the round's first sweep; later sweeps read their list length and
        // first entry after the grid barrier, with the end-of-round test
        s_len = ld_acquire(&ctl->list_len[s0 % kListSlots]);
        s_tile = (rk >= 0 && (uint32_t)rk < s_len) ? take_entry_b(p.lists + (size_t)(s0 % kListSlots) * MT, (uint32_t)rk) : -1;
        s_done_t = -1;
    }
    __syncthreads();
    if (s_dec[0] == -3) return;   // a wait ran out (recorded)

    // one thread: publish the done stamp of the last visited tile (release:
    // the visit's writes, block barriers before, come with it)
    auto publish_done = [&]() {
        const int dt = s_done_t;
        if (dt >= 0) {
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p.done + dt), "r"(s_done_v) : "memory");
            s_done_t = -1;
        }
    };
    auto hook = [&]() {
        if (threadIdx.x == 32) publish_done();
    };
    // one visit of global tile t in sweep sv (an entry outside its grid's
    // tile range, which the queue never holds, is skipped); returns the
    // visit's first layer
    auto visit = [&](int t, uint32_t sv, uint32_t *fmask, unsigned *lastj, uint32_t *slot_out,
                     const MazeDesc **dout, int *ty, int *tx, bool with_hook) {
        const uint32_t slot = __ldg(p.tile_maze + t);
        const MazeDesc &dref = p.descs[slot];
        // defensive: a list entry must lie in its grid's tile range
        const bool valid = (uint32_t)t - dref.tile_base < (uint32_t)(dref.ntx * dref.nty);
        wave::Visit v;
        v.g = dref.g;
        v.dist_bits = dref.dist_bits;
        v.TY = dref.TY;
        v.TXW = dref.TXW;
        v.k = dref.k;
        const int ntx = dref.ntx;
        const uint32_t local = (uint32_t)t - dref.tile_base;
        v.ty = (int)(local / (uint32_t)ntx);
        v.tx = (int)(local - (uint32_t)v.ty * ntx);
        v.l0 = (sv - dref.start_sweep) * (uint32_t)v.k;
        const uint32_t maxl = dref.max_layers;
        v.jmax = v.k;
        if (maxl && v.l0 + (uint32_t)v.k > maxl) v.jmax = (int)(maxl - v.l0);
        v.par = (int)(sv & 1u);
        *fmask = 0u;
        *lastj = 0u;
        if (valid) {
            if (with_hook) wave::visit_tile<RXW, R, NW, WPL>(v, sm, &p.descs[slot].err, fmask, lastj, wave::LogSink(), nullptr, hook);
            else wave::visit_tile<RXW, R, NW, WPL>(v, sm, &p.descs[slot].err, fmask, lastj);
        }
        if (maxl && v.l0 + (uint32_t)v.k >= maxl) *fmask = 0u;   // fixed depth reached
        *slot_out = slot;
        *dout = &dref;
        *ty = v.ty;
        *tx = v.tx;
        return v.l0;
    };

    for (uint32_t s = s0;; ++s) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && s > s0) {
            // list slot (s + 3) % 4 last served sweep s - 1 and next serves s + 3
            const uint32_t r = (s + 3) % kListSlots;
            ctl->work[r] = 0u;
            ctl->list_len[r] = 0u;
        }
        uint32_t *list = p.lists + (size_t)(s % kListSlots) * MT;
        unsigned *work = &ctl->work[s % kListSlots];
        const uint32_t len = s_len;
        // lookahead (and the done stamps it reads) only where the sweep has
        // more than a quarter as many tiles as blocks: a tail of visits to fill
        const bool la_s = p.lookahead && len > G / 4;
        int t = s_tile;
        if (t < 0 && threadIdx.x == 0) {
            // (a list no longer than the grid has no entries past the blocks' own)
            const uint32_t i = pend_mine >= 0 ? (uint32_t)pend_mine : (len > G ? G + atomicAdd(work, 1u) : len);
            pend_mine = -1;
            s_tile = (i < len) ? take_entry_b(list, i) : -1;
        }
        __syncthreads();
        t = s_tile;
        const uint32_t stamp = s + 2u;            // queued for sweep s + 1
        const uint32_t sl1 = (s + 1u) % kListSlots;
        uint32_t *stamps1 = p.stamps + (size_t)((s + 1u) % kStampSlots) * MT;
        int64_t pend_gt = -1;                     // lanes 0..8: global tile of a push in flight
        uint32_t pend_old = 0u, pend_slot = 0u;   // its stamp before the atomicMax, its grid
        while (t >= 0) {
            uint32_t next_i = 0;
            vq ^= 1u;
            if (threadIdx.x == 0) {
                if (pend_mine >= 0) {
                    next_i = (uint32_t)pend_mine;
                    pend_mine = -1;
                } else {
                    next_i = len > G ? G + atomicAdd(work, 1u) : len;
                }
                s_mask[vq] = 0u;
                s_lastj[vq] = 0u;
            }
            uint32_t fmask, slot;
            unsigned lastj;
            const MazeDesc *dp;
            int ty, tx;
            const uint32_t l0 = visit(t, s, &fmask, &lastj, &slot, &dp, &ty, &tx, la_s);
            uint32_t pend_i = 0u;
            const bool pend_new = pend_gt >= 0 && pend_old < stamp;   // previous visit's push
            if (pend_new) pend_i = atomicAdd(&ctl->list_len[sl1], 1u);
            if (fmask) atomicOr(&s_mask[vq], fmask);
            if (lastj) atomicMax(&s_lastj[vq], lastj);
            if (threadIdx.x == 0) {
                ++blk_visits;
                s_tile = (next_i < len) ? take_entry_b(list, next_i) : -1;
            }
            __syncthreads();
            if (threadIdx.x == 0 && la_s) {
                s_done_t = t;   // published by the next visit's hook, or before the block waits
                s_done_v = s + 1u;
            }
            if (threadIdx.x < 9) {
                if (pend_new) {
                    wave::st_relaxed(p.lists + (size_t)sl1 * MT + pend_i, (uint32_t)pend_gt + 1u);
                    atomicMax(&p.descs[pend_slot].last_push, stamp);
                }
                // this visit's push for border zone threadIdx.x: stamp now, append later
                const uint32_t zone = 1u << threadIdx.x;
                pend_gt = (s_mask[vq] & zone) ? zone_tile_b(*dp, ty, tx, zone) : -1;
                if (pend_gt >= 0) {
                    pend_slot = slot;
                    pend_old = atomicMax(stamps1 + pend_gt, stamp);
                }
                if (threadIdx.x == 0 && s_lastj[vq]) atomicMax(&p.descs[slot].maxl, l0 + s_lastj[vq]);
            }
            t = s_tile;
        }
        if (pend_gt >= 0 && pend_old < stamp) {   // the sweep's last visit
            const uint32_t i = atomicAdd(&ctl->list_len[sl1], 1u);
            wave::st_relaxed(p.lists + (size_t)sl1 * MT + i, (uint32_t)pend_gt + 1u);
            atomicMax(&p.descs[pend_slot].last_push, stamp);
        }

        // ---- end of sweep s: arrive, then run ready tiles of sweep s + 1
        // until every block has arrived ----
        const unsigned target = (s + 1 - s0) * G;
        __syncthreads();
        if (threadIdx.x == 0) {
            publish_done();
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
        }
        const bool last = p.round_sweeps && s + 1 - s0 >= p.round_sweeps;   // the round's last sweep
        const bool look = la_s && !last;
        uint32_t *list1 = p.lists + (size_t)sl1 * MT;
        const uint32_t *stamps0 = p.stamps + (size_t)(s % kStampSlots) * MT;
        bool fixed_taken = false;   // thread 0: this block's first entry of s + 1 ran
        unsigned spins = 0;         // thread 0: idle polls
        int toggle = 0;
        for (unsigned it = 0;; it ^= 1u) {
            if (warp == 0) {
                int dec = -2, cand = -1, cidx = -1;
                if (lane == 0) {
                    int fe = -1, me = -1;
                    if (look) {
                        if (!fixed_taken) fe = (int)ld_relaxed(list1 + rk) - 1;
                        if (pend_mine >= 0 && (uint32_t)pend_mine < MT) me = (int)ld_relaxed(list1 + pend_mine) - 1;
                    }
                    if (ld_acquire(&ctl->bar_count) >= target) {
                        dec = -1;
                    } else if (look) {
                        if (fe >= 0 && (me < 0 || !toggle)) {
                            cand = fe;
                            cidx = rk;
                        } else if (me >= 0) {
                            cand = me;
                            cidx = pend_mine;
                        }
                        toggle ^= 1;
                        if (pend_mine < 0 && (fixed_taken || fe < 0 || toggle))
                            pend_mine = (int)(G + atomicAdd(&ctl->work[sl1], 1u));
                    }
                }
                dec = __shfl_sync(0xffffffffu, dec, 0);
                cand = __shfl_sync(0xffffffffu, cand, 0);
                if (dec == -2 && cand >= 0) {
                    // lanes 0..8: has the neighbour (in the candidate's grid) that
                    // sweep s still had to visit finished it?
                    bool ok = true;
                    if (lane < 9) {
                        const MazeDesc &cd = p.descs[__ldg(p.tile_maze + cand)];
                        const uint32_t local = (uint32_t)cand - cd.tile_base;
                        const int cy = (int)(local / (uint32_t)cd.ntx), cx = (int)(local - (uint32_t)cy * cd.ntx);
                        const int ny = cy + lane / 3 - 1, nx = cx + lane % 3 - 1;
                        if (local < (uint32_t)(cd.ntx * cd.nty) && ny >= 0 && nx >= 0 && ny < cd.nty && nx < cd.ntx) {
                            const uint32_t n = cd.tile_base + (uint32_t)(ny * cd.ntx + nx);
                            const uint32_t st = ld_relaxed(stamps0 + n), dn = ld_acquire(p.done + n);
                            ok = st != s + 1u || dn >= s + 1u;
                        }
                    }
                    if (__all_sync(0xffffffffu, ok)) {
                        dec = cand;
                        if (lane == 0) {
                            wave::st_relaxed(list1 + cidx, 0u);
                            if (cidx == rk && !fixed_taken) fixed_taken = true;
                            else pend_mine = -1;
                        }
                    }
                }
                if (lane == 0) {
                    if (dec == -2) {
                        ++spins;
                        if ((spins & 63u) == 0u && (ld_acquire(&ctl->err) & ERR_TIMEOUT)) dec = -3;
                        if (spins > p.spin_limit) {
                            atomicOr(&ctl->err, ERR_TIMEOUT);
                            dec = -3;
                        }
                        if (dec == -2 && spins > 8) __nanosleep(32);
                    }
                    s_dec[it] = dec;   // (read two polls ago, before the last block barrier)
                }
            }
            __syncthreads();
            const int d = s_dec[it];
            if (d == -3) return;   // a wait ran out (recorded): every block stops
            if (d == -1) break;    // every block has arrived
            if (d == -2) continue;
            // ---- a visit of global tile d in sweep s + 1 ----
            vq ^= 1u;
            if (threadIdx.x == 0) {
                s_mask[vq] = 0u;
                s_lastj[vq] = 0u;
            }
            uint32_t fmask, slot;
            unsigned lastj;
            const MazeDesc *dp;
            int ty, tx;
            const uint32_t l1 = visit(d, s + 1u, &fmask, &lastj, &slot, &dp, &ty, &tx, false);
            if (fmask) atomicOr(&s_mask[vq], fmask);
            if (lastj) atomicMax(&s_lastj[vq], lastj);
            if (threadIdx.x == 0) ++blk_visits;
            __syncthreads();
            if (threadIdx.x == 0) {
                s_done_t = d;
                s_done_v = s + 2u;
                publish_done();   // the block waits anyway: out at once
                spins = 0;
            }
            if (threadIdx.x < 9) {   // what it reaches goes to sweep s + 2 at once
                const uint32_t zone = 1u << threadIdx.x;
                if (s_mask[vq] & zone) {
                    const int64_t gt2 = zone_tile_b(*dp, ty, tx, zone);
                    if (gt2 >= 0) push_gt_b(p, slot, (uint32_t)gt2, s + 2u);
                }
                if (threadIdx.x == 0 && s_lastj[vq]) atomicMax(&p.descs[slot].maxl, l1 + s_lastj[vq]);
            }
        }

        if (threadIdx.x == 0) {
            // one read gives the end-of-round test and the next sweep's list
            // length; the block's own entry of it comes alongside
            const uint32_t nlen = ld_relaxed(&ctl->list_len[sl1]);
            const uint32_t fe = fixed_taken ? 0u : ld_relaxed(list1 + rk);
            const unsigned done = (nlen == 0u) || last;
            if (done && blockIdx.x == 0) {
                p.bc->next_sweep = s + 1;
                ctl->sweeps = s + 1 - s0;
                // list slots the next round pushes into start empty; its first
                // list (s + 1) is kept, with a fresh claim counter
                for (uint32_t q = 0; q < (uint32_t)kListSlots; ++q) {
                    ctl->work[q] = 0u;
                    if (q != sl1) ctl->list_len[q] = 0u;
                }
            }
            if (done && blk_visits) atomicAdd(&ctl->visits, blk_visits);
            s_done = done;
            s_len = nlen;
            int first = -1;
            if (!done) {   // (a finished round leaves list s + 1 to the next round)
                if (!fixed_taken && (uint32_t)rk < nlen && fe) {
                    first = (int)fe - 1;
                    wave::st_relaxed(list1 + rk, 0u);
                }
                if (first < 0 && pend_mine >= 0) {
                    if ((uint32_t)pend_mine < nlen) first = take_entry_b(list1, (uint32_t)pend_mine);
                    pend_mine = -1;
                }
                if (pend_mine >= 0 && (uint32_t)pend_mine >= nlen) pend_mine = -1;   // never written
            }
            s_tile = first;
        }
        __syncthreads();
        if (s_done) return;
    }
}

// ---- per-grid mode: every grid keeps its own sweep clock ----
//
// A ticket is 1 + a global tile id. The tickets of a grid's sweep s are
// published together once its sweep s - 1 has finished (by the block that
// finished its last visit), into ring 0 if the sweep has at most kFlowSmall
// tiles, else ring 1; blocks take ring 0 first. So a grid never waits for
// another grid's sweep, and a grid with few tiles per sweep (a maze) is not
// queued behind the many tiles of a large one. Exactness is the same as with
// one clock for all grids: a sweep's visits read their halos as of the start
// of the sweep (parity of the grid's own sweep), and no visit of sweep s + 1
// of a grid starts before every visit of its sweep s has finished.

__device__ __forceinline__ uint64_t flow_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0: claim a ticket; the global tile id, -1 once no grid of the round
// is active (then no ticket is out), -2 after a wait ran out (recorded). A
// claim is a fetch-and-add on the ring's head, taken only when the ring holds
// unclaimed tickets; a block that lost the race for the last of them keeps
// its index and waits for the ring's next publication to fill it (or for the
// round to end: no grid active and the index past the ring's final tail).
// (A compare-and-swap claim lost most races under hundreds of claimers: one
// winner per round trip.) Both waits end after 30 s of the global timer in
// which nothing was published.
__device__ int flow_claim(const BatchParams &p, BatchCtl *bc) {
    unsigned spins = 0, nap = 32;
    uint64_t idle0 = flow_ns();
    uint32_t seen = 0xffffffffu;   // tails last seen (their sum grows with every publication)
    for (;;) {
        uint32_t tsum = 0u;
        for (int r = 0; r < 2; ++r) {
            const uint32_t t = ld_acquire(&bc->tail[r].v);
            tsum += t;
            if (ld_relaxed(&bc->head[r].v) >= t) continue;
            const uint32_t h = atomicAdd(&bc->head[r].v, 1u);
            uint32_t *e = p.ring + (size_t)r * (p.ring_mask + 1u) + (h & p.ring_mask);
            uint64_t t0 = flow_ns();
            uint32_t seen_r = t;
            for (unsigned w = 1;; ++w) {
                const uint32_t v = ld_acquire(e);
                if (v) {
                    wave::st_relaxed(e, 0u);
                    return (int)(v - 1u);
                }
                if ((w & 15u) == 0u) {
                    const uint32_t tr = ld_acquire(&bc->tail[r].v);
                    if (ld_acquire(&bc->active.v) == 0u && tr <= h) return -1;
                    if (ld_acquire(&bc->c.err) & ERR_TIMEOUT) return -2;
                    if (tr != seen_r) {   // the ring moves on: the wait is not stuck
                        seen_r = tr;
                        t0 = flow_ns();
                    } else if (flow_ns() - t0 > 30000000000ull) {   // 30 s without a publication
                        atomicOr(&bc->c.err, ERR_TIMEOUT);
                        return -2;
                    }
                }
                __nanosleep(w < 16 ? 32 : 256);
            }
        }
        ++spins;
        if ((spins & 7u) == 0u && ld_acquire(&bc->active.v) == 0u) return -1;
        if (tsum != seen) {   // something was published since the last look
            seen = tsum;
            idle0 = flow_ns();
        }
        if ((spins & 63u) == 0u) {
            if (ld_acquire(&bc->c.err) & ERR_TIMEOUT) return -2;
            if (flow_ns() - idle0 > 30000000000ull) {   // 30 s without a publication
                atomicOr(&bc->c.err, ERR_TIMEOUT);
                return -2;
            }
        }
        __nanosleep(nap);   // idle: poll less often the longer nothing comes
        if (nap < 512) nap *= 2;
    }
}

// Store ticket `v` at index `i` of ring r once the slot's previous ticket has
// been taken (bounded wait; false after spin_limit polls, recorded).
__device__ __forceinline__ bool flow_put(const BatchParams &p, BatchCtl *bc, uint32_t r, uint32_t i,
                                         uint32_t v, unsigned spin_limit) {
    uint32_t *e = p.ring + (size_t)r * (p.ring_mask + 1u) + (i & p.ring_mask);
    unsigned w = 0;
    while (ld_acquire(e) != 0u) {
        if (++w > spin_limit) {
            atomicOr(&bc->c.err, ERR_TIMEOUT);
            return false;
        }
        if (w > 8) __nanosleep(32);
    }
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(e), "r"(v) : "memory");
    return true;
}

template <int RXW, int R, int NW, int MINB, int WPL = 1>
__global__ void __launch_bounds__(NW * 32, MINB) k_batch_flow(BatchParams p) {
    __shared__ wave::VisitSmem<RXW, NW, WPL> sm;
    __shared__ int s_tile;
    __shared__ unsigned s_mask, s_lastj;
    __shared__ uint32_t s_pub_n, s_pub_base, s_pub_r;
    BatchCtl *bc = p.bc;
    Ctl *ctl = &bc->c;
    const size_t MT = p.max_tiles;
    unsigned long long blk_visits = 0;
    sm.zero_pad();   // (the first barrier below publishes it)
    for (;;) {
        if (threadIdx.x == 0) {
            s_mask = 0u;
            s_lastj = 0u;
            s_tile = flow_claim(p, bc);
        }
        __syncthreads();
        const int t = s_tile;
        if (t < 0) break;   // block-uniform
        // ---- one visit of tile t at its grid's current sweep ----
        const uint32_t slot = __ldg(p.tile_maze + t);
        MazeDesc &dref = p.descs[slot];
        const uint32_t ls = ld_relaxed(&dref.ls);   // fixed while this sweep's tickets are out
        wave::Visit v;
        v.g = dref.g;
        v.dist_bits = dref.dist_bits;
        v.TY = dref.TY;
        v.TXW = dref.TXW;
        v.k = dref.k;
        const uint32_t local = (uint32_t)t - dref.tile_base;
        const bool valid = local < (uint32_t)(dref.ntx * dref.nty);   // defensive
        v.ty = (int)(local / (uint32_t)dref.ntx);
        v.tx = (int)(local - (uint32_t)v.ty * dref.ntx);
        v.l0 = ls * (uint32_t)v.k;
        const uint32_t maxl = dref.max_layers;
        v.jmax = v.k;
        if (maxl && v.l0 + (uint32_t)v.k > maxl) v.jmax = (int)(maxl - v.l0);
        v.par = (int)(ls & 1u);
        uint32_t fmask = 0u;
        unsigned lastj = 0u;
        if (valid) wave::visit_tile<RXW, R, NW, WPL>(v, sm, &dref.err, &fmask, &lastj);
        if (maxl && v.l0 + (uint32_t)v.k >= maxl) fmask = 0u;   // fixed depth reached
        if (fmask) atomicOr(&s_mask, fmask);
        if (lastj) atomicMax(&s_lastj, lastj);
        if (threadIdx.x == 0) ++blk_visits;
        __syncthreads();
        // ---- the tiles it reaches, queued for the grid's sweep ls + 1: lanes
        // 0..8 of warp 0 (one border zone each), one count-up for all ----
        if (threadIdx.x < 32) {
            const uint32_t zone = 1u << threadIdx.x;
            int64_t gt = -1;
            if (threadIdx.x < 9 && (s_mask & zone)) gt = zone_tile_b(dref, v.ty, v.tx, zone);
            const bool fresh = gt >= 0 && atomicMax(p.stamps + gt, ls + 2u) < ls + 2u;
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            if (fm) {
                const int lead = __ffs(fm) - 1;
                const uint32_t q1 = (ls + 1u) & 1u;
                uint32_t base = 0u;
                if ((int)threadIdx.x == lead) base = atomicAdd(&dref.cnt[q1], (uint32_t)__popc(fm));
                base = __shfl_sync(0xffffffffu, base, lead);
                if (fresh)
                    wave::st_relaxed(p.lists + (size_t)q1 * MT + dref.tile_base + base +
                                         (uint32_t)__popc(fm & ((1u << threadIdx.x) - 1u)),
                                     (uint32_t)gt + 1u);
            }
            if (threadIdx.x == 0 && s_lastj) atomicMax(&dref.maxl, v.l0 + s_lastj);
        }
        __syncthreads();   // the visit's writes and pushes come before the count-down
        // ---- count down the grid's sweep; the last visit moves the grid on ----
        if (threadIdx.x == 0) {
            s_pub_n = 0u;
            uint32_t old;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                         : "=r"(old) : "l"(&dref.pend), "r"(0xffffffffu) : "memory");
            if (old == 1u) {
                const uint32_t q1 = (ls + 1u) & 1u;
                const uint32_t n = ld_relaxed(&dref.cnt[q1]);
                const uint32_t ran = ls + 1u - dref.ls0;
                atomicMax(&ctl->sweeps, ran);
                // with a sweep budget B: a grid counts as reached once it ran B
                // sweeps (or converged before); it pauses once every grid of
                // the round has reached B, or at 16 B -- so a grid of fast
                // sweeps is not held to a slow grid's pace within the round
                const uint32_t B = p.round_sweeps;
                if (B && (ran == B || (n == 0u && ran < B))) atomicAdd(&bc->reached.v, 1u);
                const bool pause = B && n != 0u &&
                                   (ran >= 16u * B || (ran >= B && ld_acquire(&bc->reached.v) >= bc->round_grids));
                if (n == 0u || pause) {
                    // converged, or paused (its next sweep's list is
                    // published by the next round)
                    dref.ls = ls + 1u;
                    dref.fstate = n == 0u ? kFlowDone : kFlowReady;
                    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&bc->active.v),
                                 "r"(0xffffffffu) : "memory");
                } else {
                    dref.ls = ls + 1u;
                    dref.pend = n;
                    dref.cnt[q1] = 0u;   // (the entries stay; slot q1 serves sweep ls + 3 next)
                    const uint32_t r = n <= kFlowSmall ? 0u : 1u;
                    s_pub_base = atomicAdd(&bc->tail[r].v, n);
                    s_pub_r = r;
                    s_pub_n = n;
                }
            }
        }
        __syncthreads();
        const uint32_t pn = s_pub_n;
        if (pn) {   // block-uniform: publish sweep ls + 1's tickets
            const uint32_t q1 = (ls + 1u) & 1u;
            const uint32_t *lst = p.lists + (size_t)q1 * MT + dref.tile_base;
            for (uint32_t i = threadIdx.x; i < pn; i += blockDim.x)
                if (!flow_put(p, bc, s_pub_r, s_pub_base + i, ld_relaxed(lst + i), p.spin_limit)) break;
        }
    }
    if (threadIdx.x == 0 && blk_visits) atomicAdd(&ctl->visits, blk_visits);
}

// Per-grid mode, round preparation: fresh rings and counters ...
__global__ void k_flow_reset(BatchCtl *bc) {
    bc->c.err = 0u;
    bc->c.sweeps = 0u;
    bc->head[0].v = bc->head[1].v = 0u;
    bc->tail[0].v = bc->tail[1].v = 0u;
    bc->active.v = 0u;
    bc->reached.v = 0u;
    bc->round_grids = 0u;
}

// ... then, one warp per grid slot, the first sweep of every grid that is
// ready (new, or paused at the last round's budget) published.
__global__ void k_flow_prep(BatchParams p, uint32_t nslots) {
    const int lane = threadIdx.x & 31;
    const uint32_t slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (slot >= nslots) return;
    MazeDesc &d = p.descs[slot];
    if (d.fstate != kFlowReady) return;   // warp-uniform
    const uint32_t q = d.ls & 1u, n = d.cnt[q];
    uint32_t base = 0u, r = n <= kFlowSmall ? 0u : 1u;
    if (lane == 0) {
        if (n) {
            base = atomicAdd(&p.bc->tail[r].v, n);
            d.pend = n;
            d.cnt[q] = 0u;
            d.ls0 = d.ls;
            d.fstate = kFlowRun;
            atomicAdd(&p.bc->active.v, 1u);
            atomicAdd(&p.bc->round_grids, 1u);
        } else {
            d.fstate = kFlowDone;   // (a grid always has its targets' tiles queued)
        }
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    const uint32_t *lst = p.lists + (size_t)q * p.max_tiles + d.tile_base;
    uint32_t *ring = p.ring + (size_t)r * (p.ring_mask + 1u);
    for (uint32_t i = lane; i < n; i += 32) ring[(base + i) & p.ring_mask] = lst[i];
}

// Submit-time check: every target in range and on a free cell, every start
// in range (bit 0: target out of range, 1: target on an obstacle, 2: start
// out of range).
__global__ void k_check_inputs(const uint32_t *free_bits, int H, int W, int P,
                               const uint32_t *targets, int nt, const uint32_t *starts, int ns,
                               uint32_t *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t N = (uint64_t)H * W;
    if (i < nt) {
        const uint32_t t = targets[i];
        if (t >= N) {
            atomicOr(flag, 1u);
        } else {
            const int y = (int)(t / (uint32_t)W), x = (int)(t % (uint32_t)W);
            if (!((free_bits[(size_t)y * P + (x >> 5)] >> (x & 31)) & 1u)) atomicOr(flag, 2u);
        }
    }
    if (i < ns && starts[i] >= N) atomicOr(flag, 4u);
}

// Round preparation on the device, so that the round itself has fixed
// launch parameters and can be replayed from a CUDA graph: a fresh claim
// counter for the round's first sweep and a clear error word.
__global__ void k_round_prep(BatchCtl *bc) {
    const uint32_t s = bc->next_sweep;
    bc->c.work[s % kListSlots] = 0u;
    bc->c.err = 0u;
    bc->c.bar_count = 0u;   // the round's barriers count from zero
}

__global__ void k_fill_u32(uint32_t *p, uint32_t n, uint32_t v) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = v;
}

template <int RXW, int R, int NW, int MINB, int WPL = 1>
void *batch_ptr() {
    return (void *)k_batch_propagate<RXW, R, NW, MINB, WPL>;
}

template <int RXW, int R, int NW, int MINB, int WPL = 1>
void *flow_ptr() {
    return (void *)k_batch_flow<RXW, R, NW, MINB, WPL>;
}

void *flow_fn(int v) {
    switch (v) {
        case 0: return flow_ptr<8, 4, 8, 3>();
        case 1: return flow_ptr<8, 8, 8, 2>();
        case 12: return flow_ptr<8, 4, 4, 4, 2>();
        default: return nullptr;
    }
}

// The batch runs on compiled shape 0 (128-row x 8-word region), its 256-row
// sibling 1, or shape 12 (the same region held by 4 warps of two words x four
// rows per lane); per grid only the depth varies.
void *batch_fn(int v) {
    switch (v) {
        case 0: return batch_ptr<8, 4, 8, 3>();
        case 1: return batch_ptr<8, 8, 8, 2>();
        case 12: return batch_ptr<8, 4, 4, 4, 2>();
        default: return nullptr;
    }
}

// ---- host side --------------------------------------------------------

constexpr size_t kAlign = 256;
size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, capacity) (offsets in bytes or tile ids).
struct RangeAlloc {
    std::map<size_t, size_t> free_;   // offset -> length
    size_t capacity = 0, used = 0;
    void init(size_t cap) {
        capacity = cap;
        used = 0;
        free_.clear();
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        if (!n) return;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// Admitted: waiting for its first round. Running: in flight. Traced: done
// (paths in the arena, or traced on demand by mpn_batch_result when they did
// not fit). Failed: done with an error.
enum class MState { Admitted, Running, Traced, Failed };

struct HostMaze {
    uint64_t ticket = 0;
    uint32_t slot = 0;
    int H = 0, W = 0, P = 0, dist_bits = 32;
    int ntx = 0, nty = 0, TY = 0, TXW = 0, k = 32;
    uint32_t tile_base = 0, ntiles = 0;
    uint32_t max_layers = 0;
    int nt = 0, ns = 0;
    // arena blocks: planes (freed after tracing) and results (kept)
    size_t planes_off = 0, planes_bytes = 0;
    size_t res_off = 0, res_bytes = 0;       // dist + targets + starts + offsets + status
    size_t cells_off = 0, cells_bytes = 0;
    size_t dist_o = 0, tgt_o = 0, st_o = 0, off_o = 0, sts_o = 0;   // within the result block
    MState state = MState::Admitted;
    mpn_status code = MPN_OK;
    uint32_t layers = 0;
    uint64_t total = 0;
    bool has_tiles = false, has_planes = false;
    bool paths_ready = false;   // cells traced into the arena
};

}  // namespace
}  // namespace mpn

using namespace mpn;

struct mpn_batch {
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    int variant = 0, blocks = 0;
    int depth_override = 0;
    uint32_t max_slots = 0, max_tiles = 0;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    RangeAlloc mem, tiles;
    MazeDesc *d_descs = nullptr;
    uint32_t *d_tile_maze = nullptr, *d_stamps = nullptr, *d_done = nullptr, *d_lists = nullptr;
    BatchCtl *d_bc = nullptr;
    uint32_t *d_rank = nullptr;       // block-rank counters, zeroed before every round
    SeedJob *d_jobs = nullptr;
    MazeDesc *h_descs = nullptr;      // pinned mirror for readback
    BatchCtl *h_bc = nullptr;         // pinned
    SeedJob *h_jobs = nullptr;        // pinned
    uint32_t *h_flag = nullptr;       // pinned
    std::vector<uint32_t> free_slots;
    std::map<uint64_t, HostMaze> mazes;
    uint64_t next_ticket = 1;
    uint32_t next_sweep = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the paths of the grids a round finished are measured and walked
    // together: a job per grid, the walks' lengths and order (grown on demand,
    // outside the arena budget)
    WalkJob *d_wjobs = nullptr, *h_wjobs = nullptr;
    uint64_t *d_totals = nullptr, *h_totals = nullptr;
    uint32_t *d_walk_len = nullptr, *d_order = nullptr;
    size_t walk_cap = 0;
    // walks longer than kLongWalk: a jump table (one grid at a time) and the
    // segments of all of them (grown on demand, outside the arena budget)
    uint32_t *d_jump = nullptr;
    size_t jump_cells = 0;
    BatchSeg *d_segs = nullptr;   // followed by the segment counter
    size_t seg_cap = 0;
    std::map<uint64_t, cudaGraphExec_t> graphs;   // one captured round per (max_sweeps, mode, lookahead)
    bool use_graph = true;
    // per-grid mode (mpn_batch_set_mode): every grid keeps its own sweep clock
    bool flow = false;
    int flow_blocks = 0;
    uint32_t *d_ring = nullptr;   // two ticket rings
    uint32_t ring_mask = 0;
    float last_round_ms = 0.f;
    uint64_t rounds = 0, sweeps_total = 0;
};

namespace {

mpn_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return MPN_OK;
    note_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? MPN_ENOMEM : MPN_ECUDA;
}

#define B_TRY(expr)                                   \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return cuda_st(e_);    \
    } while (0)

bool dev_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void *arena_at(mpn_batch *b, size_t off) { return (char *)b->arena + off; }

// Depth used for a grid: the override if set, else the autotuner's pick for
// its size bucket and the batch's tile shape, else 32.
int depth_for(mpn_batch *b, int H, int W) {
    if (b->depth_override) return b->depth_override;
    int d = 0;
    if (tune_lookup(H, W, b->variant, &d)) return d;   // the autotuner's pick for this size
    return 32;
}

void release_planes(mpn_batch *b, HostMaze &m) {
    if (m.has_planes) {
        b->mem.release(m.planes_off, m.planes_bytes);
        m.has_planes = false;
    }
    if (m.has_tiles) {
        b->tiles.release(m.tile_base, m.ntiles);
        m.has_tiles = false;
    }
}

}  // namespace

extern "C" {

mpn_status mpn_batch_create(uint64_t budget_bytes, int32_t variant, void *stream, mpn_batch **out) {
    if (!out || budget_bytes < (1u << 20)) return MPN_EINVAL;
    *out = nullptr;
    if (variant < 0) variant = 0;
    if (!batch_fn(variant)) return MPN_EINVAL;
    mpn_batch *b = new (std::nothrow) mpn_batch();
    if (!b) return MPN_ENOMEM;
    b->stream = (cudaStream_t)stream;
    b->variant = variant;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    const VariantDesc vd = variant_desc(variant);
    int bps = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_fn(variant), vd.nwarps * 32, 0);
    if (e != cudaSuccess || bps < 1) {
        delete b;
        return e == cudaSuccess ? MPN_ECUDA : cuda_st(e);
    }
    b->blocks = bps * b->sm_count;
    b->max_slots = 4096;
    // a tile covers at least 32 x 192 cells (>= ~27 KB of planes at uint32)
    size_t mt = budget_bytes / 8192;
    if (mt > (1u << 22)) mt = 1u << 22;
    if (mt < 4096) mt = 4096;
    b->max_tiles = (uint32_t)mt;
    b->arena_bytes = budget_bytes;
    e = cudaMalloc(&b->arena, budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_descs, b->max_slots * sizeof(MazeDesc));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_tile_maze, (size_t)b->max_tiles * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_stamps, (size_t)b->max_tiles * kStampSlots * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_done, (size_t)b->max_tiles * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_lists, (size_t)b->max_tiles * kListSlots * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_bc, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_rank, kRankWords * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_jobs, b->max_slots * sizeof(SeedJob));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_descs, b->max_slots * sizeof(MazeDesc));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_bc, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_jobs, b->max_slots * sizeof(SeedJob));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_flag, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_stamps, 0, (size_t)b->max_tiles * kStampSlots * 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, (size_t)b->max_tiles * 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_lists, 0, (size_t)b->max_tiles * kListSlots * 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bc, 0, sizeof(BatchCtl), b->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_wjobs, b->max_slots * sizeof(WalkJob));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_wjobs, b->max_slots * sizeof(WalkJob));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_totals, 2 * b->max_slots * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_totals, 2 * b->max_slots * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        mpn_batch_destroy(b);
        return cuda_st(e);
    }
    b->mem.init(budget_bytes);
    b->tiles.init(b->max_tiles);
    for (uint32_t i = b->max_slots; i-- > 0;) b->free_slots.push_back(i);
    // per-grid sweep clocks by default (the shape has that kernel)
    if (flow_fn(variant)) {
        const mpn_status ms = mpn_batch_set_mode(b, 1);
        if (ms != MPN_OK) {
            mpn_batch_destroy(b);
            return ms;
        }
    }
    *out = b;
    return MPN_OK;
}

mpn_status mpn_batch_set_mode(mpn_batch *b, int32_t per_grid_clock) {
    if (!b || (per_grid_clock != 0 && per_grid_clock != 1)) return MPN_EINVAL;
    if (!b->mazes.empty()) return MPN_ESTATE;   // only while the batch holds no grid
    if (!per_grid_clock) {
        b->flow = false;
        return MPN_OK;
    }
    void *fn = flow_fn(b->variant);
    if (!fn) return MPN_EINVAL;
    const VariantDesc vd = variant_desc(b->variant);
    int bps = 0;
    B_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, vd.nwarps * 32, 0));
    if (bps < 1) return MPN_ECUDA;
    if (!b->d_ring) {
        // each ring holds every tile of the batch once plus a claim per block
        size_t n = 1;
        while (n < (size_t)b->max_tiles + (size_t)bps * b->sm_count + 1) n <<= 1;
        B_TRY(cudaMalloc((void **)&b->d_ring, 2 * n * sizeof(uint32_t)));
        B_TRY(cudaMemsetAsync(b->d_ring, 0, 2 * n * sizeof(uint32_t), b->stream));
        B_TRY(cudaStreamSynchronize(b->stream));
        b->ring_mask = (uint32_t)(n - 1);
    }
    b->flow_blocks = bps * b->sm_count;
    b->flow = true;
    return MPN_OK;
}

mpn_status mpn_batch_set_depth(mpn_batch *b, int32_t depth) {
    if (!b || depth < 0 || depth > 32) return MPN_EINVAL;
    const VariantDesc vd = variant_desc(b->variant);
    const int ry = region_rows(vd);
    if (depth && ry - 2 * depth < depth) return MPN_EINVAL;
    b->depth_override = depth;
    return MPN_OK;
}

mpn_status mpn_batch_submit(mpn_batch *b, const uint8_t *mask, int32_t H, int32_t W,
                            const uint32_t *targets, int32_t nt, const uint32_t *starts, int32_t ns,
                            int32_t dist_bits, uint32_t max_layers, uint64_t *ticket) {
    NvtxRange nvtx_range("mpn_batch_submit");
    if (!b || !mask || !targets || nt < 1 || ns < 0 || (ns > 0 && !starts) || !ticket) return MPN_EINVAL;
    if (H < 1 || W < 1 || (uint64_t)H * W >= 0xffffffffull) return MPN_EINVAL;
    if (dist_bits == MPN_DIST_AUTO) dist_bits = ((int64_t)H * W <= 65535) ? 16 : 32;
    if (dist_bits != 16 && dist_bits != 32) return MPN_EINVAL;
    if (b->free_slots.empty()) return MPN_ENOMEM;
    HostMaze m;
    m.H = H;
    m.W = W;
    m.P = (((W + 31) / 32) + 3) / 4 * 4;
    m.dist_bits = dist_bits;
    m.k = depth_for(b, H, W);
    const VariantDesc vd = variant_desc(b->variant);
    const int ry = region_rows(vd);
    m.TY = ry - 2 * m.k;
    m.TXW = vd.rxw - 2;
    m.ntx = ((W + 31) / 32 + m.TXW - 1) / m.TXW;
    m.nty = (H + m.TY - 1) / m.TY;
    m.ntiles = (uint32_t)(m.ntx * m.nty);
    m.max_layers = max_layers;
    m.nt = nt;
    m.ns = ns;
    const size_t plane = align_up((size_t)H * m.P * 4);
    m.planes_bytes = 5 * plane;   // free bits + propagation state (4 words per word)
    m.dist_o = 0;
    m.tgt_o = align_up((size_t)H * W * (dist_bits / 8));
    m.st_o = m.tgt_o + align_up((size_t)nt * 4);
    m.off_o = m.st_o + align_up((size_t)(ns > 0 ? ns : 1) * 4);
    m.sts_o = m.off_o + align_up((size_t)(ns + 1) * 8);
    m.res_bytes = m.sts_o + align_up((size_t)(ns > 0 ? ns : 1));
    // admission by device memory: planes + results must fit now, tiles too
    size_t tb = 0;
    if (!b->tiles.alloc(m.ntiles, &tb)) return MPN_ENOMEM;
    if (!b->mem.alloc(m.planes_bytes, &m.planes_off)) {
        b->tiles.release(tb, m.ntiles);
        return MPN_ENOMEM;
    }
    if (!b->mem.alloc(m.res_bytes, &m.res_off)) {
        b->tiles.release(tb, m.ntiles);
        b->mem.release(m.planes_off, m.planes_bytes);
        return MPN_ENOMEM;
    }
    m.tile_base = (uint32_t)tb;
    m.has_tiles = m.has_planes = true;
    m.slot = b->free_slots.back();
    b->free_slots.pop_back();
    m.ticket = b->next_ticket++;

    // inputs into the arena (host or device sources), planes initialised
    cudaStream_t st = b->stream;
    char *res = (char *)arena_at(b, m.res_off);
    uint32_t *fb = (uint32_t *)arena_at(b, m.planes_off);
    cudaError_t e = cudaSuccess;
    const cudaMemcpyKind kt = dev_ptr(targets) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = cudaMemcpyAsync(res + m.tgt_o, targets, (size_t)nt * 4, kt, st);
    if (e == cudaSuccess && ns > 0)
        e = cudaMemcpyAsync(res + m.st_o, starts, (size_t)ns * 4,
                            dev_ptr(starts) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    // a host mask is staged in the (not yet filled) distance plane, which is
    // at least H*W bytes
    const uint8_t *dmask = mask;
    if (e == cudaSuccess && !dev_ptr(mask)) {
        dmask = (const uint8_t *)(res + m.dist_o);
        e = cudaMemcpyAsync((void *)dmask, mask, (size_t)H * W, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = launch_pack(dmask, H, W, m.P, fb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync((char *)fb + plane, 0, 4 * plane, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(res + m.dist_o, 0xff, (size_t)H * W * (dist_bits / 8), st);
    // reject bad end-points now, so that no grid can fail while in flight
    uint32_t *flag = (uint32_t *)((char *)fb + plane);   // one word of the zeroed state
    if (e == cudaSuccess) {
        const int n = nt > ns ? nt : ns;
        count_launch();
        k_check_inputs<<<(n + 255) / 256, 256, 0, st>>>(fb, H, W, m.P, (const uint32_t *)(res + m.tgt_o),
                                                        nt, (const uint32_t *)(res + m.st_o), ns, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_flag, flag, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mpn_status bad = MPN_OK;
    if (e == cudaSuccess && *b->h_flag) bad = (*b->h_flag & 2u) && !(*b->h_flag & 5u) ? MPN_EOBSTACLE : MPN_EINVAL;
    if (e != cudaSuccess || bad != MPN_OK) {
        release_planes(b, m);
        b->mem.release(m.res_off, m.res_bytes);
        b->free_slots.push_back(m.slot);
        return e != cudaSuccess ? cuda_st(e) : bad;
    }
    b->mazes.emplace(m.ticket, m);
    *ticket = m.ticket;
    return MPN_OK;
}

// The round: device-side preparation, then the cooperative persistent launch.
static cudaError_t enqueue_round(mpn_batch *b, const BatchParams &p) {
    cudaStream_t st = b->stream;
    cudaError_t e;
    if (b->flow) {   // fresh rings, then every ready grid's first sweep published
        k_flow_reset<<<1, 1, 0, st>>>(b->d_bc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_flow_prep<<<(b->max_slots + 7) / 8, 256, 0, st>>>(p, b->max_slots);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else {
        k_round_prep<<<1, 1, 0, st>>>(b->d_bc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(b->d_rank, 0, kRankWords * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    // external records, so that they time the round also when it is captured
    e = cudaEventRecordWithFlags(b->ev0, st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    const VariantDesc vd = variant_desc(b->variant);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->flow ? b->flow_blocks : b->blocks);
    cfg.blockDim = dim3(vd.nwarps * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BatchParams pp = p;
    void *args[] = {&pp};
    e = cudaLaunchKernelExC(&cfg, b->flow ? flow_fn(b->variant) : batch_fn(b->variant), args);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags(b->ev1, st, cudaEventRecordExternal);
}

// Run one round from a CUDA graph captured the first time this max_sweeps
// value is used (launch parameters are fixed: everything that changes from
// round to round lives in device memory).
static cudaError_t run_round(mpn_batch *b, const BatchParams &p) {
    if (!b->use_graph) {
        count_launch(2);
        return enqueue_round(b, p);
    }
    const uint64_t key = ((uint64_t)p.round_sweeps << 2) | ((uint64_t)b->flow << 1) | (p.lookahead & 1u);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        cudaStream_t keep = b->stream;
        b->stream = cs;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_round(b, p);
            e = cudaStreamEndCapture(cs, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        b->stream = keep;
        cudaStreamDestroy(cs);
        cudaGraphExec_t ge = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            // capture not available: run rounds as plain launches from now on
            cudaGetLastError();
            b->use_graph = false;
            count_launch(2);
            return enqueue_round(b, p);
        }
        it = b->graphs.emplace(key, ge).first;
    }
    count_launch(2);
    return cudaGraphLaunch(it->second, b->stream);
}

static cudaError_t launch_batch_trace(mpn_batch *b, const HostMaze &m, uint32_t *cells,
                                      cudaStream_t st) {
    char *res = (char *)arena_at(b, m.res_off);
    GridDev g;
    g.free_bits = nullptr;
    g.state = nullptr;
    g.dist = res + m.dist_o;
    g.H = m.H;
    g.W = m.W;
    g.P = m.P;
    return launch_trace(g, m.dist_bits, (const uint32_t *)(res + m.st_o), m.ns,
                        (const uint64_t *)(res + m.off_o), (const int8_t *)(res + m.sts_o), cells,
                        nullptr, st, &b->d_bc->c.err);
}

// Wait for the stream, then trace every grid that converged in the last round.
static mpn_status finish_round(mpn_batch *b) {
    NvtxRange nvtx_range("mpn_batch_finish_round");
    cudaStream_t st = b->stream;
    B_TRY(cudaMemcpyAsync(b->h_bc, b->d_bc, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
    B_TRY(cudaMemcpyAsync(b->h_descs, b->d_descs, b->max_slots * sizeof(MazeDesc),
                          cudaMemcpyDeviceToHost, st));
    B_TRY(cudaStreamSynchronize(st));
    b->next_sweep = b->h_bc->next_sweep;
    if (b->h_bc->c.err & ERR_TIMEOUT) {
        // (per-grid mode: tickets may be left in the rings; start them empty)
        if (b->flow) cudaMemsetAsync(b->d_ring, 0, 2 * ((size_t)b->ring_mask + 1) * sizeof(uint32_t), st);
        return MPN_ETIMEOUT;
    }
    std::vector<HostMaze *> done;
    for (auto &kv : b->mazes) {
        HostMaze &m = kv.second;
        if (m.state != MState::Running) continue;
        const MazeDesc &d = b->h_descs[m.slot];
        if (b->flow ? d.fstate != kFlowDone                    // per-grid mode: not converged yet
                    : d.last_push > b->next_sweep) continue;   // tiles still queued for the next sweep
        if (d.err) {
            // (a uint16 overflow; end-points were checked at submit) -- the grid
            // has drained, so its planes can go
            m.state = MState::Failed;
            m.code = (d.err & ERR_OVERFLOW) ? MPN_EOVERFLOW : MPN_ECUDA;
            release_planes(b, m);
            continue;
        }
        {
            m.layers = d.maxl;
            done.push_back(&m);
        }
    }
    if (done.empty()) return MPN_OK;
    // one walk job per newly converged grid: status, lengths, offsets and
    // totals of all of them in one launch, then one wait
    Ctl *ctl = &b->d_bc->c;
    const int nj = (int)done.size();
    uint64_t nwalks = 0;
    for (HostMaze *m : done) nwalks += (uint64_t)m->ns;
    if (nwalks >= 0xffffffffull) return MPN_EINVAL;
    if (nwalks > b->walk_cap) {
        size_t cap = b->walk_cap ? b->walk_cap : (1u << 16);
        while (cap < nwalks) cap *= 2;
        cudaFree(b->d_walk_len);
        cudaFree(b->d_order);
        b->d_walk_len = b->d_order = nullptr;
        b->walk_cap = 0;
        B_TRY(cudaMalloc((void **)&b->d_walk_len, cap * sizeof(uint32_t)));
        B_TRY(cudaMalloc((void **)&b->d_order, cap * sizeof(uint32_t)));
        b->walk_cap = cap;
    }
    uint32_t base = 0;
    for (int j = 0; j < nj; ++j) {
        const HostMaze *m = done[j];
        char *res = (char *)arena_at(b, m->res_off);
        WalkJob &jb = b->h_wjobs[j];
        jb.g.free_bits = (const uint32_t *)arena_at(b, m->planes_off);
        jb.g.state = nullptr;
        jb.g.dist = res + m->dist_o;
        jb.g.H = m->H;
        jb.g.W = m->W;
        jb.g.P = m->P;
        jb.starts = (const uint32_t *)(res + m->st_o);
        jb.offsets = (uint64_t *)(res + m->off_o);
        jb.status = (int8_t *)(res + m->sts_o);
        jb.cells = nullptr;
        jb.dist_bits = m->dist_bits;
        jb.ns = (uint32_t)m->ns;
        jb.walk_base = base;
        jb.split = 0;
        base += (uint32_t)m->ns;
    }
    B_TRY(cudaMemcpyAsync(b->d_wjobs, b->h_wjobs, nj * sizeof(WalkJob), cudaMemcpyHostToDevice, st));
    B_TRY(launch_batch_lengths(b->d_wjobs, nj, b->d_walk_len, b->d_totals, &ctl->err, st));
    B_TRY(cudaMemcpyAsync(b->h_totals, b->d_totals, 2 * nj * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    B_TRY(cudaStreamSynchronize(st));
    // the bit planes are not needed any more (walks read the distances);
    // paths of every finished grid whose paths fit in the arena now, walked
    // together, longest first; the others are traced on demand into the
    // caller's buffer
    bool any = false;
    for (int j = 0; j < nj; ++j) {
        HostMaze *m = done[j];
        m->total = b->h_totals[j];
        m->state = MState::Traced;
        release_planes(b, *m);
        m->cells_bytes = align_up((size_t)(m->total ? m->total : 1) * 4);
        if (!b->mem.alloc(m->cells_bytes, &m->cells_off)) {
            m->cells_bytes = 0;
            continue;
        }
        b->h_wjobs[j].cells = (uint32_t *)arena_at(b, m->cells_off);
        m->paths_ready = true;
        any = any || m->total > 0;
    }
    if (!any) return MPN_OK;
    // grids with walks far longer than the rest: those walks are cut into
    // segments (first cells from a jump table), walked side by side
    uint64_t segs_needed = 0;
    size_t jump_need = 0;
    for (int j = 0; j < nj; ++j) {
        const HostMaze *m = done[j];
        if (!b->h_wjobs[j].cells || b->h_totals[nj + j] <= kLongWalk) continue;
        segs_needed += m->total / kSegLen + (uint64_t)m->ns + 1;
        jump_need = std::max(jump_need, (size_t)m->H * m->W);
    }
    bool split = segs_needed > 0 && segs_needed < 0xffffffffull;
    if (split && jump_need > b->jump_cells) {
        cudaFree(b->d_jump);
        b->d_jump = nullptr;
        b->jump_cells = 0;
        if (cudaMalloc((void **)&b->d_jump, 2 * jump_need * sizeof(uint32_t)) == cudaSuccess) b->jump_cells = jump_need;
        else cudaGetLastError();
    }
    if (split && segs_needed > b->seg_cap) {
        cudaFree(b->d_segs);
        b->d_segs = nullptr;
        b->seg_cap = 0;
        if (cudaMalloc((void **)&b->d_segs, segs_needed * sizeof(BatchSeg) + 16) == cudaSuccess) b->seg_cap = segs_needed;
        else cudaGetLastError();
    }
    split = split && b->jump_cells >= jump_need && b->seg_cap >= segs_needed;   // else: walked whole
    uint32_t *nseg = split ? (uint32_t *)(b->d_segs + b->seg_cap) : nullptr;
    if (split)
        for (int j = 0; j < nj; ++j)
            if (b->h_wjobs[j].cells && b->h_totals[nj + j] > kLongWalk) b->h_wjobs[j].split = 1;
    B_TRY(cudaMemcpyAsync(b->d_wjobs, b->h_wjobs, nj * sizeof(WalkJob), cudaMemcpyHostToDevice, st));
    if (split) {
        B_TRY(cudaMemsetAsync(nseg, 0, sizeof(uint32_t), st));
        for (int j = 0; j < nj; ++j) {
            const WalkJob &jb = b->h_wjobs[j];
            if (!jb.split) continue;
            uint32_t *table = nullptr;
            B_TRY(launch_jump_table(jb.g, jb.dist_bits, b->d_jump, &table, st));
            B_TRY(launch_batch_segments(b->d_wjobs, j, jb.ns, jb.dist_bits, table, b->d_segs,
                                        (uint32_t)b->seg_cap, nseg, &ctl->err, st));
        }
        B_TRY(launch_batch_segwalks(b->d_wjobs, b->d_segs, nseg, (uint32_t)segs_needed, &ctl->err, st));
    }
    B_TRY(launch_batch_walks(b->d_wjobs, nj, b->d_walk_len, (uint32_t)nwalks, b->d_order, &ctl->err, st));
    // a walk that found no cell one step closer (not a distance plane)
    B_TRY(cudaMemcpyAsync(&b->h_bc->c.err, &ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    B_TRY(cudaStreamSynchronize(st));
    if (b->h_bc->c.err & ERR_TRACE) return MPN_ECUDA;
    return MPN_OK;
}

mpn_status mpn_batch_run(mpn_batch *b, uint32_t max_sweeps, int32_t *n_running, int32_t *n_done) {
    NvtxRange nvtx_range("mpn_batch_run");
    if (!b) return MPN_EINVAL;
    cudaStream_t st = b->stream;
    // descriptors and seeds of the grids admitted since the last round
    int njobs = 0;
    for (auto &kv : b->mazes) {
        HostMaze &m = kv.second;
        if (m.state != MState::Admitted) continue;
        MazeDesc d{};
        char *res = (char *)arena_at(b, m.res_off);
        const size_t plane = m.planes_bytes / 5;
        d.g.free_bits = (const uint32_t *)arena_at(b, m.planes_off);
        d.g.state = (uint32_t *)((char *)arena_at(b, m.planes_off) + plane);
        d.g.dist = res + m.dist_o;
        d.g.H = m.H;
        d.g.W = m.W;
        d.g.P = m.P;
        d.dist_bits = m.dist_bits;
        d.ntx = m.ntx;
        d.nty = m.nty;
        d.TY = m.TY;
        d.TXW = m.TXW;
        d.k = m.k;
        d.tile_base = m.tile_base;
        d.start_sweep = b->next_sweep;
        d.max_layers = m.max_layers;
        d.fstate = b->flow ? kFlowReady : kFlowIdle;   // (ls, pend, cnt start at zero)
        b->h_descs[m.slot] = d;
        B_TRY(cudaMemcpyAsync(b->d_descs + m.slot, &b->h_descs[m.slot], sizeof(MazeDesc),
                              cudaMemcpyHostToDevice, st));
        b->h_jobs[njobs].slot = m.slot;
        b->h_jobs[njobs].n = (uint32_t)m.nt;
        b->h_jobs[njobs].targets = (const uint32_t *)(res + m.tgt_o);
        ++njobs;
        m.state = MState::Running;
    }
    // tile -> slot map of the new grids
    for (int j = 0; j < njobs; ++j) {
        const HostMaze *m = nullptr;
        for (auto &kv : b->mazes)
            if (kv.second.slot == b->h_jobs[j].slot && kv.second.state == MState::Running) m = &kv.second;
        if (!m) continue;
        // queue stamps and done stamps of its tile range start at zero (the
        // range may have served an earlier grid)
        for (int q = 0; q < kStampSlots; ++q)
            B_TRY(cudaMemsetAsync(b->d_stamps + (size_t)q * b->max_tiles + m->tile_base, 0,
                                  (size_t)m->ntiles * 4, st));
        B_TRY(cudaMemsetAsync(b->d_done + m->tile_base, 0, (size_t)m->ntiles * 4, st));
        const unsigned nb = (m->ntiles + 255) / 256;
        count_launch();
        k_fill_u32<<<nb < 1024 ? nb : 1024, 256, 0, st>>>(b->d_tile_maze + m->tile_base, m->ntiles, m->slot);
        B_TRY(cudaGetLastError());
    }
    BatchParams p{};
    p.descs = b->d_descs;
    p.tile_maze = b->d_tile_maze;
    p.stamps = b->d_stamps;
    p.done = b->d_done;
    p.lists = b->d_lists;
    p.max_tiles = b->max_tiles;
    p.bc = b->d_bc;
    p.rank = b->d_rank;
    p.ring = b->d_ring;
    p.ring_mask = b->ring_mask;
    p.round_sweeps = max_sweeps;
    p.spin_limit = 1u << 24;
    p.lookahead = 1;
    // (test hook: MPN_TEST_NO_LOOKAHEAD=1 makes blocks only wait at a sweep's end)
    if (const char *ev = getenv("MPN_TEST_NO_LOOKAHEAD")) p.lookahead = (ev[0] == '1') ? 0u : 1u;
    if (njobs > 0) {
        B_TRY(cudaMemcpyAsync(b->d_jobs, b->h_jobs, njobs * sizeof(SeedJob), cudaMemcpyHostToDevice, st));
        count_launch();
        k_batch_seed<<<njobs, 128, 0, st>>>(p, b->d_jobs, b->flow ? 1u : 0u);
        B_TRY(cudaGetLastError());
    }
    int running = 0;
    for (auto &kv : b->mazes) running += kv.second.state == MState::Running;
    if (running > 0) B_TRY(run_round(b, p));
    mpn_status s = finish_round(b);
    if (running > 0) {
        if (cudaEventElapsedTime(&b->last_round_ms, b->ev0, b->ev1) != cudaSuccess) {
            cudaGetLastError();   // leave no stale error for the next launch check
            b->last_round_ms = 0.f;
        }
        b->rounds++;
        b->sweeps_total += b->h_bc->c.sweeps;
    }
    int r = 0, d = 0;
    for (auto &kv : b->mazes) {
        r += kv.second.state == MState::Running || kv.second.state == MState::Admitted;
        d += kv.second.state == MState::Traced || kv.second.state == MState::Failed;
    }
    if (n_running) *n_running = r;
    if (n_done) *n_done = d;
    return s;
}

mpn_status mpn_batch_poll(mpn_batch *b, uint64_t ticket, int32_t *state) {
    if (!b || !state) return MPN_EINVAL;
    auto it = b->mazes.find(ticket);
    if (it == b->mazes.end()) return MPN_EINVAL;
    const MState s = it->second.state;
    *state = s == MState::Traced ? MPN_BATCH_DONE : s == MState::Failed ? MPN_BATCH_FAILED
                                                                        : MPN_BATCH_PENDING;
    return s == MState::Failed ? it->second.code : MPN_OK;
}

mpn_status mpn_batch_wait(mpn_batch *b, uint64_t ticket, uint32_t max_sweeps, int32_t *state) {
    if (!b) return MPN_EINVAL;
    int32_t s = MPN_BATCH_PENDING;
    for (uint32_t round = 0; round < (1u << 20); ++round) {
        const mpn_status ps = mpn_batch_poll(b, ticket, &s);
        if (s != MPN_BATCH_PENDING || (ps != MPN_OK && s != MPN_BATCH_FAILED)) {
            if (state) *state = s;
            return ps;
        }
        int32_t running = 0, done = 0;
        const mpn_status rs = mpn_batch_run(b, max_sweeps, &running, &done);
        if (rs != MPN_OK) {
            if (state) *state = s;
            return rs;
        }
    }
    if (state) *state = s;
    return MPN_ETIMEOUT;
}

mpn_status mpn_batch_result(mpn_batch *b, uint64_t ticket, void *dist, uint64_t *offsets,
                            uint32_t *cells, uint64_t cells_cap, int8_t *status, uint32_t *layers) {
    NvtxRange nvtx_range("mpn_batch_result");
    if (!b) return MPN_EINVAL;
    auto it = b->mazes.find(ticket);
    if (it == b->mazes.end()) return MPN_EINVAL;
    HostMaze &m = it->second;
    if (m.state == MState::Failed) return m.code;
    if (m.state != MState::Traced) return MPN_ESTATE;
    cudaStream_t st = b->stream;
    char *res = (char *)arena_at(b, m.res_off);
    auto kind = [](const void *p) {
        return dev_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    };
    if (layers) *layers = m.layers;
    if (dist)
        B_TRY(cudaMemcpyAsync(dist, res + m.dist_o, (size_t)m.H * m.W * (m.dist_bits / 8), kind(dist), st));
    if (offsets)
        B_TRY(cudaMemcpyAsync(offsets, res + m.off_o, (size_t)(m.ns + 1) * 8, kind(offsets), st));
    if (status && m.ns > 0)
        B_TRY(cudaMemcpyAsync(status, res + m.sts_o, (size_t)m.ns, kind(status), st));
    if (cells && m.total > 0) {
        if (m.total > cells_cap) {
            B_TRY(cudaStreamSynchronize(st));
            return MPN_ENOMEM;
        }
        if (m.paths_ready) {
            B_TRY(cudaMemcpyAsync(cells, arena_at(b, m.cells_off), (size_t)m.total * 4, kind(cells), st));
        } else if (dev_ptr(cells)) {
            B_TRY(launch_batch_trace(b, m, cells, st));            // straight into the caller's buffer
        } else {
            // host buffer and no room in the arena: a temporary device buffer
            void *tmp = nullptr;
            B_TRY(cudaMalloc(&tmp, (size_t)m.total * 4));
            cudaError_t e = launch_batch_trace(b, m, (uint32_t *)tmp, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cells, tmp, (size_t)m.total * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            cudaFree(tmp);
            B_TRY(e);
        }
    }
    B_TRY(cudaStreamSynchronize(st));
    return MPN_OK;
}

mpn_status mpn_batch_info(mpn_batch *b, uint64_t ticket, int32_t *H, int32_t *W, int32_t *dist_bits,
                          uint64_t *total_cells) {
    if (!b) return MPN_EINVAL;
    auto it = b->mazes.find(ticket);
    if (it == b->mazes.end()) return MPN_EINVAL;
    const HostMaze &m = it->second;
    if (H) *H = m.H;
    if (W) *W = m.W;
    if (dist_bits) *dist_bits = m.dist_bits;
    if (total_cells) *total_cells = m.total;
    return MPN_OK;
}

mpn_status mpn_batch_release(mpn_batch *b, uint64_t ticket) {
    if (!b) return MPN_EINVAL;
    auto it = b->mazes.find(ticket);
    if (it == b->mazes.end()) return MPN_EINVAL;
    HostMaze &m = it->second;
    if (m.state == MState::Running || m.state == MState::Admitted) return MPN_ESTATE;
    release_planes(b, m);
    b->mem.release(m.res_off, m.res_bytes);
    if (m.cells_bytes) b->mem.release(m.cells_off, m.cells_bytes);
    b->free_slots.push_back(m.slot);
    b->mazes.erase(it);
    return MPN_OK;
}

mpn_status mpn_batch_stats(mpn_batch *b, mpn_batch_stats_t *out) {
    if (!b || !out) return MPN_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->arena_bytes = b->arena_bytes;
    out->arena_used = b->mem.used;
    out->tiles_used = b->tiles.used;
    out->next_sweep = b->next_sweep;
    out->rounds = b->rounds;
    out->sweeps = b->sweeps_total;
    out->last_round_ms = b->last_round_ms;
    out->blocks = b->blocks;
    out->graph = b->use_graph ? 1 : 0;
    for (auto &kv : b->mazes) {
        const MState s = kv.second.state;
        out->admitted += s == MState::Admitted;
        out->running += s == MState::Running;
        out->done += s == MState::Traced;
        out->failed += s == MState::Failed;
    }
    return MPN_OK;
}

void mpn_batch_destroy(mpn_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    cudaFree(b->arena);
    cudaFree(b->d_descs);
    cudaFree(b->d_tile_maze);
    cudaFree(b->d_stamps);
    cudaFree(b->d_done);
    cudaFree(b->d_lists);
    cudaFree(b->d_bc);
    cudaFree(b->d_rank);
    cudaFree(b->d_ring);
    cudaFree(b->d_jobs);
    if (b->h_descs) cudaFreeHost(b->h_descs);
    if (b->h_bc) cudaFreeHost(b->h_bc);
    if (b->h_jobs) cudaFreeHost(b->h_jobs);
    if (b->h_flag) cudaFreeHost(b->h_flag);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    cudaFree(b->d_wjobs);
    cudaFree(b->d_totals);
    cudaFree(b->d_walk_len);
    cudaFree(b->d_order);
    cudaFree(b->d_jump);
    cudaFree(b->d_segs);
    if (b->h_wjobs) cudaFreeHost(b->h_wjobs);
    if (b->h_totals) cudaFreeHost(b->h_totals);
    delete b;
}

}  // extern "C"
