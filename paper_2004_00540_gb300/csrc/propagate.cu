// Activity propagation for one grid: the stack of max-pool layers (Methods,
// "Activity Map Generation", Fig. 1) on bit planes (see wave.cuh for why a
// layer is a 1-bit dilation).
//
// k_propagate is persistent and temporally blocked: the grid is cut into tiles;
// a tile visit loads the tile plus a halo of k rows and one word (32 cells) on
// each side into registers and advances k layers there, then writes back the
// interior. Sweeps of k layers are separated by a grid-wide barrier; inside a
// sweep only tiles that the frontier can reach within k layers are visited:
// a visit that ends with frontier cells queues the tiles they can reach for
// the next sweep, and blocks claim work from that list.
//
// k_plain_layer is the paper's recursive mode (Appendix, Table I), one launch
// per layer over the whole distance plane, kept as the baseline.
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "mpn_internal.cuh"
#include "wave.cuh"

namespace mpn {

namespace {

using wave::ld_acquire;
using wave::ld_relaxed;
using wave::border_bits;

// Queue tile (ty, tx) for sweep s unless it is queued already (one entry per
// tile per sweep: the sweep's stamp only grows). The entry holds 1 + the tile
// id; a block that waits at the end of the previous sweep may poll it.
__device__ __forceinline__ void push_tile(const PropParams &p, int ty, int tx, uint32_t s) {
    if (ty < 0 || tx < 0 || ty >= p.nty || tx >= p.ntx) return;
    const int t = ty * p.ntx + tx;
    const size_t ntl = (size_t)p.ntx * p.nty;
    if (atomicMax(p.stamps + (size_t)(s % kStampSlots) * ntl + t, s + 1) < s + 1) {
        const uint32_t slot = s % kListSlots;
        const uint32_t i = atomicAdd(&p.ctl->list_len[slot], 1u);
        wave::st_relaxed(p.lists + (size_t)slot * ntl + i, (uint32_t)t + 1u);
    }
}

// Take entry i of a tile list: the tile id (-1 if the entry was never
// written), and clear the entry for the list slot's next use.
__device__ __forceinline__ int take_entry(uint32_t *list, uint32_t i) {
    const uint32_t e = ld_relaxed(list + i);
    if (e) wave::st_relaxed(list + i, 0u);
    return (int)e - 1;
}

// Queue every tile that frontier cells in these border zones of tile
// (ty, tx) can reach within k layers.
__device__ void push_reached(const PropParams &p, int ty, int tx, uint32_t zones, uint32_t s) {
    if (zones & FB_ANY) push_tile(p, ty, tx, s);
    if (zones & FB_N) push_tile(p, ty - 1, tx, s);
    if (zones & FB_S) push_tile(p, ty + 1, tx, s);
    if (zones & FB_W) push_tile(p, ty, tx - 1, s);
    if (zones & FB_E) push_tile(p, ty, tx + 1, s);
    if (zones & FB_NW) push_tile(p, ty - 1, tx - 1, s);
    if (zones & FB_NE) push_tile(p, ty - 1, tx + 1, s);
    if (zones & FB_SW) push_tile(p, ty + 1, tx - 1, s);
    if (zones & FB_SE) push_tile(p, ty + 1, tx + 1, s);
}

// The tile that frontier cells in border zone z (one FB_* bit) of tile
// (ty, tx) can reach, or -1 past the grid's edge.
__device__ __forceinline__ int zone_tile(const PropParams &p, int ty, int tx, uint32_t z) {
    if (z & (FB_N | FB_NW | FB_NE)) --ty;
    if (z & (FB_S | FB_SW | FB_SE)) ++ty;
    if (z & (FB_W | FB_NW | FB_SW)) --tx;
    if (z & (FB_E | FB_NE | FB_SE)) ++tx;
    if (ty < 0 || tx < 0 || ty >= p.nty || tx >= p.ntx) return -1;
    return ty * p.ntx + tx;
}

// Persistent temporally blocked propagation over one grid (tile shapes: see
// wave::visit_tile). A visit's queue pushes are split across the next visit:
// lanes 0..8 (one border zone each) issue the stamp's atomicMax after the
// visit, and append the tile to the list once the next visit's layers are
// done, so neither atomic's round trip stands between two visits; the last
// visit of a sweep finishes its pushes before the grid barrier.
//
// Lookahead at the end of a sweep: a block that has arrived at the grid
// barrier of sweep s does not only wait. It takes entries of sweep s + 1's
// list (its own first entry, then entries claimed with the counter) and runs
// a tile as soon as every tile of its 3 x 3 neighbourhood that sweep s still
// had to visit has finished that visit (stamps and done[] say which): the
// tile's region then holds exactly the state at the start of sweep s + 1,
// which is what the visit must read, so the result is the same as after the
// barrier. Such a visit queues what it reaches for sweep s + 2 at once.
template <int RXW, int R, int NW, int MINB, typename DT, int WPL = 1>
__global__ void __launch_bounds__(NW * 32, MINB) k_propagate(PropParams p) {
    static_assert(RXW == 4 || RXW == 8 || RXW == 16 || RXW == 32, "region words");
    static_assert(R >= 1, "rows per lane");
    __shared__ wave::VisitSmem<RXW, NW, WPL> sm;
    __shared__ int s_tile;
    __shared__ unsigned s_mask[2], s_done, s_maxl, s_ok;   // s_mask by visit parity
    __shared__ uint32_t s_len;                              // length of this sweep's list
    __shared__ int s_chunk;                                 // activation-log chunk, -1: none
    __shared__ unsigned s_cursor;                           // entries used in it
    __shared__ int s_dec[2];   // end of sweep, by poll parity: -3 stop, -2 wait, -1 go on, >= 0 run tile

    const int ntiles = p.ntx * p.nty;
    Ctl *ctl = p.ctl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned thr_maxl = 0u;              // largest layer this thread's words reached
    unsigned long long blk_visits = 0;   // thread 0: tile visits of this block
    unsigned long long blk_layers = 0;   // thread 0: layers those visits ran
    unsigned vq = 0u;                    // visit parity (block-uniform)
    bool log_more = p.log != nullptr;    // thread 0: the pool may still have chunks
    const uint32_t maxv = (uint32_t)(p.TY * p.TXW) + 1u;   // log entries one visit can need
    unsigned hdr = 0u;                   // thread 0: this visit's header slot in the chunk
    uint32_t prev_head = 0u;             // thread 0: the tile's latest header before it
    uint32_t prev_nv = 0u;               // thread 0: the tile's logged visits before it
    unsigned long long blk_entries = 0;  // thread 0: word entries this block logged
    const wave::LogSink lg{p.log, &s_chunk, &s_cursor};
    int pend_mine = -1;                  // thread 0: list index claimed while waiting, not yet run
    __shared__ int s_done_t;             // visited tile whose done stamp is not out yet (-1: none)
    __shared__ uint32_t s_done_v;        // its stamp

    sm.zero_pad();   // (the first barrier below publishes it)
    // the seeding step rejected the targets (nothing in this kernel sets these
    // bits, so every block takes the same branch)
    if (ld_acquire(&ctl->err) & (ERR_INVAL | ERR_OBSTACLE)) return;

    wave::Visit v;
    v.g = p.g;
    v.dist_bits = sizeof(DT) * 8;
    v.TY = p.TY;
    v.TXW = p.TXW;
    v.k = p.k;
    const size_t ntl = (size_t)ntiles;
    const uint32_t G = gridDim.x;   // <= ntiles, so list + rk is inside every list
    int rk = 0;   // thread 0: this block's rank in the lists' fixed deal (wave::block_rank)
    if (threadIdx.x == 0) {
        rk = wave::block_rank(p.rank, p.spin_limit, &ctl->err);
        s_ok = rk >= 0;
        // sweep 0: entry rk of the seeded list is this block's first tile
        s_len = ld_acquire(&ctl->list_len[0]);
        s_tile = (rk >= 0 && (uint32_t)rk < s_len) ? take_entry(p.lists, (uint32_t)rk) : -1;
        s_chunk = -1;
        s_cursor = 0u;
        s_done_t = -1;
    }
    __syncthreads();
    if (!s_ok) return;   // a wait ran out (recorded)

    // thread 0, before a visit of tile t: room in the log chunk, the header
    // slot, the tile's chain so far (its previous visit has finished)
    auto log_begin = [&](int t) {
        if (log_more && (s_chunk < 0 || s_cursor + maxv > kLogChunk)) {
            // this chunk may not hold the visit's entries: take the next one
            const uint32_t c = atomicAdd(&ctl->log_next, 1u);
            log_more = c < p.log_chunks;
            s_chunk = log_more ? (int)c : -1;
            s_cursor = 0u;
        }
        if (s_chunk >= 0) {   // the header goes in front of the visit's entries
            hdr = s_cursor;
            s_cursor = hdr + 1u;
            prev_head = ld_relaxed(p.tile_head + t);
            prev_nv = ld_relaxed(p.tile_nv + t);
        }
    };
    // one thread: publish the done stamp of the last visited tile with a
    // release store, which orders the visit's writes (state, log, header;
    // block barriers between) before the stamp: a reader that sees the stamp
    // sees them.
    auto publish_done = [&]() {
        const int dt = s_done_t;
        if (dt >= 0) {
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p.done + dt), "r"(s_done_v) : "memory");
            s_done_t = -1;
        }
    };
    // during a visit's layers, thread 32 (nothing of its own in flight then,
    // so the release costs little) publishes the previous visit's stamp
    auto hook = [&]() {
        if (threadIdx.x == 32) publish_done();
    };
    // Lookahead pays only where a sweep has enough tiles to leave a tail of
    // visits to fill (more than a quarter as many as blocks, measured on the
    // 23170^2 grid and the 1024^2 maze); a sparser sweep is about one round of
    // visits side by side, so its visits publish no done stamps and its end
    // has no lookahead. (Every block decides this from the same list length.)
    bool la_s = false;
    // thread 0, after the visit's block barrier: its header (unless it logged
    // nothing: then the slot is reused); the tile's done stamp is due
    auto log_end_and_done = [&](int t, uint32_t l0v, uint32_t sweep) {
        if (s_chunk >= 0) {
            const uint32_t cnt = s_cursor - hdr - 1u;
            if (cnt) {
                const uint32_t gh = (uint32_t)s_chunk * kLogChunk + hdr;
                uint4 *h = reinterpret_cast<uint4 *>(p.log + (size_t)gh * kLogFields);
                h[0] = make_uint4(prev_head, cnt, l0v + 1u, prev_nv);
                h[1] = make_uint4(0u, 0u, 0u, 0u);
                p.tile_head[t] = gh + 1u;
                p.tile_nv[t] = prev_nv + 1u;
                if (prev_nv < kTileSlots)
                    p.tile_vis[(size_t)t * kTileSlots + prev_nv] = make_uint4(gh, cnt, l0v + 1u, 0u);
                blk_entries += cnt;
            } else {
                s_cursor = hdr;
            }
        }
        s_done_t = t;   // published by the next visit's hook, or before the block waits
        s_done_v = sweep + 1u;
    };

    for (uint32_t s = 0;; ++s) {
        const uint32_t l0 = p.l_base + s * (uint32_t)p.k;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            // list slot (s + 3) % 4 last served sweep s - 1 (no block claims
            // from it any more) and next serves sweep s + 3
            const uint32_t r = (s + 3) % kListSlots;
            ctl->work[r] = 0u;
            ctl->list_len[r] = 0u;
        }
        v.l0 = l0;
        v.jmax = p.k;
        if (p.max_layers && l0 + (uint32_t)p.k > p.max_layers) v.jmax = (int)(p.max_layers - l0);
        v.par = (int)(s & 1u);
        uint32_t *list = p.lists + (size_t)(s % kListSlots) * ntl;
        unsigned *work = &ctl->work[s % kListSlots];
        const uint32_t len = s_len;
        la_s = p.lookahead && len > G / 4;
        // entries 0..G-1 go one per block without an atomic; the rest are
        // claimed with the counter (an index claimed while waiting at the last
        // barrier comes first)
        int t = s_tile;
        if (t < 0 && threadIdx.x == 0) {
            // (a list no longer than the grid has no entries past the blocks' own)
            const uint32_t i = pend_mine >= 0 ? (uint32_t)pend_mine : (len > G ? G + atomicAdd(work, 1u) : len);
            pend_mine = -1;
            s_tile = (i < len) ? take_entry(list, i) : -1;
        }
        __syncthreads();
        t = s_tile;
        const uint32_t stamp = s + 2u;             // queued for sweep s + 1
        const uint32_t slot1 = (s + 1u) % kListSlots;
        uint32_t *stamps1 = p.stamps + (size_t)((s + 1u) % kStampSlots) * ntl;
        int pend_t = -1;                           // lanes 0..8: tile of a push in flight
        uint32_t pend_old = 0u;                    // its stamp before the atomicMax
        while (t >= 0) {
            // claim the next tile now; the atomic's latency hides behind this visit
            uint32_t next_i = 0;
            vq ^= 1u;
            if (threadIdx.x == 0) {
                if (pend_mine >= 0) {
                    next_i = (uint32_t)pend_mine;
                    pend_mine = -1;
                } else {
                    next_i = len > G ? G + atomicAdd(work, 1u) : len;
                }
                s_mask[vq] = 0u;   // last read two visits ago, before the previous visit's first barrier
                log_begin(t);
            }
            v.ty = t / p.ntx;
            v.tx = t - v.ty * p.ntx;
            uint32_t fmask;
            unsigned lastj, jrun = 0;
            if (la_s) wave::visit_tile<RXW, R, NW, WPL>(v, sm, &ctl->err, &fmask, &lastj, lg, &jrun, hook);
            else wave::visit_tile<RXW, R, NW, WPL>(v, sm, &ctl->err, &fmask, &lastj, lg, &jrun);
            uint32_t pend_i = 0u;
            const bool pend_new = pend_t >= 0 && pend_old < stamp;   // previous visit's push
            if (pend_new) pend_i = atomicAdd(&ctl->list_len[slot1], 1u);
            if (fmask) atomicOr(&s_mask[vq], fmask);
            if (lastj) thr_maxl = max(thr_maxl, l0 + lastj);
            if (threadIdx.x == 0) {
                ++blk_visits;
                blk_layers += jrun;
                s_tile = (next_i < len) ? take_entry(list, next_i) : -1;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                log_end_and_done(t, l0, s);
                if (!la_s) s_done_t = -1;   // no stamp needed
            }
            if (threadIdx.x < 9) {
                if (pend_new) wave::st_relaxed(p.lists + (size_t)slot1 * ntl + pend_i, (uint32_t)pend_t + 1u);
                // this visit's push for border zone threadIdx.x: stamp now, append later
                const uint32_t zone = 1u << threadIdx.x;
                pend_t = (s_mask[vq] & zone) ? zone_tile(p, v.ty, v.tx, zone) : -1;
                if (pend_t >= 0) pend_old = atomicMax(stamps1 + pend_t, stamp);
            }
            t = s_tile;
        }
        if (pend_t >= 0 && pend_old < stamp) {   // the sweep's last visit
            const uint32_t i = atomicAdd(&ctl->list_len[slot1], 1u);
            wave::st_relaxed(p.lists + (size_t)slot1 * ntl + i, (uint32_t)pend_t + 1u);
        }

        // ---- end of sweep s: arrive, then run ready tiles of sweep s + 1
        // until every block has arrived ----
        const unsigned target = (s + 1) * G;
        __syncthreads();
        if (threadIdx.x == 0) {
            publish_done();
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
        }
        const uint32_t l1 = l0 + (uint32_t)p.k;          // layer at the start of sweep s + 1
        const bool more = !(p.max_layers && l1 >= p.max_layers) && s + 1 < p.sweep_cap;
        const bool look = la_s && more;
        uint32_t *list1 = p.lists + (size_t)slot1 * ntl;
        const uint32_t *stamps0 = p.stamps + (size_t)(s % kStampSlots) * ntl;
        bool fixed_taken = false;                          // thread 0: this block's first entry of s + 1 ran
        unsigned spins = 0;                                // thread 0: idle polls
        int toggle = 0;                                    // thread 0: which candidate to check first
        for (unsigned it = 0;; it ^= 1u) {
            if (warp == 0) {
                int dec = -2, cand = -1, cidx = -1;
                if (lane == 0) {
                    // the candidate entries, then the barrier word with acquire
                    // (a candidate read before it is checked again below)
                    int fe = -1, me = -1;
                    if (look) {
                        if (!fixed_taken) fe = (int)ld_relaxed(list1 + rk) - 1;
                        if (pend_mine >= 0 && (uint32_t)pend_mine < ntl)
                            me = (int)ld_relaxed(list1 + pend_mine) - 1;
                    }
                    const uint32_t bc = ld_acquire(&ctl->bar_count);
                    if (bc >= target) {
                        dec = -1;
                    } else if (look) {
                        // candidates: this block's own first entry, and one claimed entry
                        if (fe >= 0 && (me < 0 || !toggle)) {
                            cand = fe;
                            cidx = rk;
                        } else if (me >= 0) {
                            cand = me;
                            cidx = pend_mine;
                        }
                        toggle ^= 1;
                        // hold one claimed entry while the own one is missing or busy
                        if (pend_mine < 0 && (fixed_taken || fe < 0 || toggle))
                            pend_mine = (int)(G + atomicAdd(&ctl->work[slot1], 1u));
                    }
                }
                dec = __shfl_sync(0xffffffffu, dec, 0);
                cand = __shfl_sync(0xffffffffu, cand, 0);
                if (dec == -2 && cand >= 0) {
                    // lanes 0..8: has the neighbour that sweep s still had to visit finished it?
                    bool ok = true;
                    if (lane < 9) {
                        const int cy = cand / p.ntx, cx = cand - cy * p.ntx;
                        const int ny = cy + lane / 3 - 1, nx = cx + lane % 3 - 1;
                        if (ny >= 0 && nx >= 0 && ny < p.nty && nx < p.ntx) {
                            const int n = ny * p.ntx + nx;
                            // (acquire: a finished visit's writes are seen with its stamp)
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
            if (d == -3) return;      // a wait ran out (recorded): every block stops
            if (d == -1) break;       // every block has arrived
            if (d == -2) continue;
            // ---- a visit of tile d in sweep s + 1 ----
            vq ^= 1u;
            if (threadIdx.x == 0) {
                s_mask[vq] = 0u;
                log_begin(d);
            }
            wave::Visit v1 = v;
            v1.l0 = l1;
            v1.jmax = p.k;
            if (p.max_layers && l1 + (uint32_t)p.k > p.max_layers) v1.jmax = (int)(p.max_layers - l1);
            v1.par = (int)((s + 1u) & 1u);
            v1.ty = d / p.ntx;
            v1.tx = d - v1.ty * p.ntx;
            uint32_t fmask;
            unsigned lastj, jrun = 0;
            wave::visit_tile<RXW, R, NW, WPL>(v1, sm, &ctl->err, &fmask, &lastj, lg, &jrun);
            if (fmask) atomicOr(&s_mask[vq], fmask);
            if (lastj) thr_maxl = max(thr_maxl, l1 + lastj);
            if (threadIdx.x == 0) {
                ++blk_visits;
                blk_layers += jrun;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                log_end_and_done(d, l1, s + 1u);
                publish_done();   // the block waits anyway: out at once
                spins = 0;
            }
            if (threadIdx.x < 9) {   // what it reaches goes to sweep s + 2 at once
                const uint32_t zone = 1u << threadIdx.x;
                if (s_mask[vq] & zone) {
                    const int nt = zone_tile(p, v1.ty, v1.tx, zone);
                    if (nt >= 0) push_tile(p, nt / p.ntx, nt - (nt / p.ntx) * p.ntx, s + 2u);
                }
            }
        }

        if (threadIdx.x == 0) {
            // decided from values no block changes before the next barrier, so
            // every block reaches the same decision; the same read gives the
            // next sweep's list length
            // (the barrier's completion was read with acquire; these two loads go out together)
            const uint32_t nlen = ld_relaxed(&ctl->list_len[slot1]);
            const uint32_t fe = fixed_taken ? 0u : ld_relaxed(list1 + rk);
            unsigned done = (nlen == 0u) || (p.max_layers && l1 >= p.max_layers);
            if (!done && s + 1 >= p.sweep_cap) {
                atomicOr(&ctl->err, ERR_SWEEPS);
                done = 1;
            }
            if (done && blockIdx.x == 0) ctl->sweeps = s + 1;
            if (done && blk_visits) {
                atomicAdd(&ctl->visits, blk_visits);
                atomicAdd(&ctl->tile_layers, blk_layers);
            }
            s_done = done;
            s_maxl = 0u;
            s_len = nlen;
            // this block's first tile of sweep s + 1: its own entry (unless it
            // ran already), else the entry it claimed while waiting
            int first = -1;
            if (!fixed_taken && (uint32_t)rk < nlen && fe) {
                first = (int)fe - 1;
                wave::st_relaxed(list1 + rk, 0u);
            }
            if (first < 0 && pend_mine >= 0) {
                if ((uint32_t)pend_mine < nlen) first = take_entry(list1, (uint32_t)pend_mine);
                pend_mine = -1;
            }
            if (pend_mine >= 0 && (uint32_t)pend_mine >= nlen) pend_mine = -1;   // never written
            s_tile = first;
        }
        __syncthreads();
        if (s_done) {
            if (thr_maxl) atomicMax(&s_maxl, thr_maxl);
            __syncthreads();
            if (threadIdx.x == 0 && s_maxl) atomicMax(&ctl->max_layer, s_maxl);
            if (threadIdx.x == 0 && blk_entries) atomicAdd(&ctl->log_entries, blk_entries);
            return;
        }
    }
}

// Distances from the activation log, after the propagation, tile by tile: a
// block takes a tile and assembles a band of its interior (all of it for the
// usual tile shapes) in shared memory, then writes the band's rows with
// coalesced stores, each cell once. The tile's visits come from its slots
// (loaded in parallel) and, past kTileSlots visits, from the chain through
// the headers, up to kDecodeBatch at a time. Each lane takes one entry
// (32-byte loads, consecutive across the warp), turns its Gray planes into
// binary planes (four XORs for all 32 cells), packs four cells' offsets as
// bytes with one multiply per plane nibble, and stores the layers of its
// reached cells into the word's 33-word row slot (the pad spreads the lanes'
// words over the banks). Entries of one word from different visits hold
// disjoint reached bits, so the order does not matter. A cell still empty
// afterwards is unreached (the unreached value, which for uint32 equals the
// empty mark) unless the propagation reached it without an entry -- a
// target, or a cell a block wrote directly once the pool ran out -- whose
// value is then read back from the plane so that it is written unchanged.
// Indices outside the pool end the tile's walk (defensive; the propagation
// never writes one).
constexpr int kDecodeBatch = 64;
static_assert(kDecodeBatch >= (int)kTileSlots && kDecodeBatch == 64,
              "the first batch holds every slot; the count prefix is two warps wide");

__device__ __forceinline__ uint32_t spread_nibble(uint32_t n) {   // bit i -> bit 8 i
    return (n * 0x204081u) & 0x01010101u;
}

// shared memory words of a band of `rows` rows: 16-bit layer codes (34 per
// word: the pad spreads a warp's words over the banks), then reached and
// covered bits per word. A tile in 32-bit mode uses half as many rows per band
// (33 words per word of cells) in the same room.
__host__ __device__ inline size_t decode_band_words(int rows, int txw) {
    return (size_t)rows * txw * 17 + 2 * (size_t)rows * txw;
}

template <typename DT, int TXW>
__global__ void __launch_bounds__(256, 6) k_log_decode(PropParams p, int band_rows, uint32_t slots) {
    extern __shared__ __align__(16) uint32_t buf[];
    __shared__ uint32_t s_gh[kDecodeBatch], s_cnt[kDecodeBatch], s_lay[kDecodeBatch];
    __shared__ uint32_t s_start[kDecodeBatch + 1];
    __shared__ uint32_t s_nvis, s_chain, s_bad, s_lo, s_narrow, s_max;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const GridDev &g = p.g;
    const int TY = p.TY;
    constexpr int CW = TXW * 32, RW = TXW * 33;   // RW: buffer words per row (32-bit mode)
    constexpr int RH = TXW * 34;                  // halves per row (16-bit mode)
    const uint32_t cap = p.log_chunks * kLogChunk;
    constexpr uint32_t kNone = 0xffffffffu;
    constexpr uint16_t kNone16 = 0xffffu, kKeep16 = 0xfffeu;
    uint16_t *b16 = reinterpret_cast<uint16_t *>(buf);
    uint32_t thr_max = 0u;   // the largest layer of this thread's log entries (the layer count L)
    if (threadIdx.x == 0) s_max = 0u;
    uint32_t *sV = buf + (size_t)band_rows * TXW * 17;    // reached bits per word
    uint32_t *sC = sV + (size_t)band_rows * TXW;          // bits covered by entries per word
    const int ntiles = p.ntx * p.nty;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty = t / p.ntx, tx = t - ty * p.ntx;
        const int ybase = ty * TY, xbase = tx * CW;
        const int rows = min(TY, g.H - ybase), cols = min(CW, g.W - xbase);
        const uint32_t nv = p.tile_nv[t];
        // slot threadIdx.x (read only below nv)
        const uint4 slot = threadIdx.x < slots ? p.tile_vis[(size_t)t * kTileSlots + threadIdx.x]
                                                    : make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();   // the previous tile's s_lo / s_narrow are no longer read
        if (threadIdx.x == 0) {
            // 16-bit codes (layer - the tile's first logged layer) when the
            // tile's layers span less than 16 bits: its first logged visit is
            // in slot 0, its last is the head of the header chain
            uint32_t lo = 0u, narrow = 1u;
            if (nv) {
                lo = slot.z;
                const uint32_t h = p.tile_head[t];
                const uint32_t hi = (h && h - 1u < cap) ? p.log[(size_t)(h - 1u) * kLogFields + 2] : lo;
                narrow = hi >= lo && (hi - lo) + 31u <= 0xfffdu;
            }
            s_lo = lo;
            s_narrow = narrow;
        }
        __syncthreads();
        const bool narrow = s_narrow != 0u;
        const uint32_t lo = s_lo;
        const int bstep = narrow ? band_rows : max(1, band_rows / 2);
        for (int b0 = 0; b0 < rows; b0 += bstep) {
            const int br = min(bstep, rows - b0);
            {
                const int n = narrow ? br * TXW * 17 : br * RW;
                uint4 *b4 = reinterpret_cast<uint4 *>(buf);
                for (int i = threadIdx.x; i < n / 4; i += 256) b4[i] = make_uint4(kNone, kNone, kNone, kNone);
                for (int i = (n & ~3) + threadIdx.x; i < n; i += 256) buf[i] = kNone;
            }
            for (int r = warp; r < br; r += 8) {
                const int gw = tx * TXW + lane;
                if (lane < TXW) {
                    sV[r * TXW + lane] = gw < g.P ? g.state[4 * ((size_t)(ybase + b0 + r) * g.P + gw)] : 0u;
                    sC[r * TXW + lane] = 0u;
                }
            }
            uint32_t done = 0;   // visits placed (block-uniform)
            if (threadIdx.x == 0) {
                s_chain = p.tile_head[t];
                s_bad = 0u;
            }
            while (done < nv) {
                // ---- gather a batch of visits: {header index, count, l0 + 1} ----
                __syncthreads();   // the previous batch's lists are no longer read
                uint32_t nb_vis;
                if (done == 0) {   // the slots (the loads went out with nv's)
                    nb_vis = min(nv, slots);
                    if (threadIdx.x < nb_vis) {
                        const uint32_t gh = slot.x;
                        s_gh[threadIdx.x] = gh;
                        s_cnt[threadIdx.x] = gh < cap ? min(slot.y, cap - gh - 1u) : 0u;
                        s_lay[threadIdx.x] = slot.z;
                    }
                } else {
                    if (threadIdx.x == 0) {
                        // the chain holds the visits past the slots, newest first
                        uint32_t n = 0u, h = s_chain;
                        const uint32_t want = min((uint32_t)kDecodeBatch, nv - done);
                        while (n < want && h != 0u && h - 1u < cap) {
                            const uint32_t gh = h - 1u;
                            const uint4 hd = *reinterpret_cast<const uint4 *>(p.log + (size_t)gh * kLogFields);
                            if (hd.w < slots) break;   // the rest sit in slots
                            s_gh[n] = gh;
                            s_cnt[n] = min(hd.y, cap - gh - 1u);
                            s_lay[n] = hd.z;
                            ++n;
                            h = hd.x;
                        }
                        s_chain = h;
                        s_bad = n < want;   // a broken chain: stop after this batch
                        s_nvis = n;
                    }
                    __syncthreads();
                    nb_vis = s_nvis;
                }
                __syncthreads();
                if (warp == 0) {   // exclusive prefix of the counts (kDecodeBatch = 2 x 32)
                    const uint32_t c0 = lane < (int)nb_vis ? s_cnt[lane] : 0u;
                    const uint32_t c1 = lane + 32 < (int)nb_vis ? s_cnt[lane + 32] : 0u;
                    uint32_t i0 = c0, i1 = c1;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint32_t u0 = __shfl_up_sync(0xffffffffu, i0, d);
                        const uint32_t u1 = __shfl_up_sync(0xffffffffu, i1, d);
                        if (lane >= d) {
                            i0 += u0;
                            i1 += u1;
                        }
                    }
                    const uint32_t tot0 = __shfl_sync(0xffffffffu, i0, 31);
                    s_start[lane] = i0 - c0;
                    s_start[lane + 32] = tot0 + i1 - c1;
                    if (lane == 31) s_start[64] = tot0 + i1;
                }
                __syncthreads();
                // ---- place the batch's entries, one per thread ----
                const uint32_t total = s_start[nb_vis];
                uint32_t vi = 0;   // visit of entry f (f only grows)
                for (uint32_t f = threadIdx.x; f < total; f += 256u) {
                    while (s_start[vi + 1] <= f) ++vi;
                    const uint4 *ep = reinterpret_cast<const uint4 *>(
                        p.log + (size_t)(s_gh[vi] + 1u + (f - s_start[vi])) * kLogFields);
                    const uint4 a = ep[0], b = ep[1];   // {pos, NB, P0, P1}, {P2, P3, P4, 0}
                    const uint32_t row = a.x / (uint32_t)TXW, word = a.x - row * (uint32_t)TXW;
                    if (row - (uint32_t)b0 >= (uint32_t)br) continue;   // another band (or bad)
                    const uint32_t nb = a.y, lay = s_lay[vi];
                    uint32_t B[5] = {a.z, a.w, b.x, b.y, b.z};
#pragma unroll
                    for (int q = 3; q >= 0; --q) B[q] ^= B[q + 1];   // Gray -> binary, bit-sliced
                    {   // the entry's last layer: a bit-sliced maximum over its reached cells
                        uint32_t cand = nb, m = 0u;
#pragma unroll
                        for (int q = 4; q >= 0; --q) {
                            const uint32_t hit = cand & B[q];
                            if (hit) {
                                m |= 1u << q;
                                cand = hit;
                            }
                        }
                        if (nb) thr_max = max(thr_max, lay + m);
                    }
                    const uint32_t w = (row - (uint32_t)b0) * (uint32_t)TXW + word;
                    atomicOr(&sC[w], nb);
                    if (narrow) {
                        uint16_t *dst = b16 + (row - (uint32_t)b0) * (uint32_t)RH + word * 34u;
                        const uint32_t l16 = lay - lo;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            uint32_t off4 = 0u;
#pragma unroll
                            for (int bb = 0; bb < 5; ++bb) off4 += spread_nibble((B[bb] >> (4 * q)) & 0xfu) << bb;
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if ((nb >> (4 * q + i)) & 1u) dst[4 * q + i] = (uint16_t)(l16 + ((off4 >> (8 * i)) & 0xffu));
                        }
                    } else {
                        uint32_t *dst = buf + (row - (uint32_t)b0) * (uint32_t)RW + word * 33u;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            uint32_t off4 = 0u;
#pragma unroll
                            for (int bb = 0; bb < 5; ++bb) off4 += spread_nibble((B[bb] >> (4 * q)) & 0xfu) << bb;
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if ((nb >> (4 * q + i)) & 1u) dst[4 * q + i] = lay + ((off4 >> (8 * i)) & 0xffu);
                        }
                    }
                }
                done += nb_vis;
                if (s_bad || nb_vis == 0) break;   // block-uniform
            }
            __syncthreads();
            // ---- reached cells without an entry keep their value (16-bit
            // mode: they are not written at all) ----
            for (int i = threadIdx.x; i < br * TXW; i += 256) {
                uint32_t m = sV[i] & ~sC[i];
                if (!m) continue;
                const int r = i / TXW, word = i - r * TXW;
                if (narrow) {
                    while (m) {
                        const int c = __ffs(m) - 1;
                        m &= m - 1u;
                        b16[r * RH + word * 34 + c] = kKeep16;
                    }
                    continue;
                }
                const DT *src = reinterpret_cast<const DT *>(g.dist) + (size_t)(ybase + b0 + r) * g.W +
                                xbase + word * 32;
                while (m) {
                    const int c = __ffs(m) - 1;
                    m &= m - 1u;
                    if (xbase + word * 32 + c < g.W) buf[r * RW + word * 33 + c] = (uint32_t)src[c];
                }
            }
            __syncthreads();
            // ---- write the band: every cell of it ----
            for (int r = warp; r < br; r += 8) {
                DT *d = reinterpret_cast<DT *>(g.dist) + (size_t)(ybase + b0 + r) * g.W + xbase + lane;
                const uint32_t *src = buf + r * RW + lane;
                const uint16_t *src16 = b16 + r * RH + lane;
#pragma unroll
                for (int w = 0; w < TXW; ++w) {   // word w: cells 32 w + lane
                    if (32 * w + lane < cols) {
                        uint32_t val;
                        if (narrow) {
                            const uint16_t c16 = src16[34 * w];
                            if (c16 == kKeep16) continue;   // reached without an entry: as it is
                            val = c16 == kNone16 ? kNone : lo + c16;
                        } else {
                            val = src[33 * w];
                        }

                        if (sizeof(DT) == 2) {
                            if (val != kNone && val > 0xfffeu) atomicOr(&p.ctl->err, ERR_OVERFLOW);
                            d[32 * w] = (DT)(val > 0xfffeu ? 0xffffu : val);
                        } else {
                            d[32 * w] = (DT)val;
                        }
                    }
                }
            }
            __syncthreads();   // before the next band or tile refills the buffer
        }
    }
    // the layer count: the largest layer of any entry (visits that wrote their
    // distances themselves counted theirs in the propagation kernel)
    const uint32_t wm = __reduce_max_sync(0xffffffffu, thr_max);
    if (lane == 0 && wm) atomicMax(&s_max, wm);
    __syncthreads();
    if (threadIdx.x == 0 && s_max) atomicMax(&p.ctl->max_layer, s_max);
}

// ---- warp-specialised variant: a producer warp stages regions with TMA ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the barrier's phase with this parity completes; false after
// ~2 s (the caller records ERR_TIMEOUT and winds down).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > 2000000000ull) return false;
    return true;
}

// 2-D tiled TMA load of the box at (x words, y rows) into shared memory,
// completing on the mbarrier (byte count).
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int y,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Block = NW consumer warps + 1 producer warp. The producer (lane 0 of the
// last warp) claims tiles, loads each claimed tile's free bits with TMA into
// one of two shared-memory buffers, and queues the tiles a finished visit
// reaches. The consumer warps take each buffer in turn, load the region's
// propagation state themselves ({V, Npar} pairs, which must be read as 64-bit
// accesses), run the tile's layers in registers (named barrier 1 only) and
// write back. So the next tile's free bits arrive while the current one is
// computed, and claims and queue pushes never stall the consumer warps. A TMA
// box starts at a word coordinate rounded down to a multiple of 4 (16-byte
// rule) and is 12 words wide; the region's 8 words start xoff = 0..3 words
// into it. Boxes outside the grid (negative or past the edge) are filled with
// zeros.
template <int RXW, int R, int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 2)
    k_propagate_tma(const __grid_constant__ CUtensorMap tm_free, PropParams p) {
    constexpr int GPW = 32 / RXW;
    constexpr int RY = NW * GPW * R;
    constexpr int BW = ((RXW + 3) + 3) / 4 * 4;   // box width in words
    constexpr uint32_t BOX_BYTES = (uint32_t)(RY * BW * 4);
    constexpr int NBAR = NW * 32;
    static_assert(RY <= 256, "TMA box height");

    __shared__ __align__(128) uint32_t sF[2][RY * BW];
    __shared__ __align__(8) uint64_t full[2], done[2];
    __shared__ int s_tile[2], s_xoff[2], s_ctile;
    __shared__ unsigned s_fmask[2], s_done, s_maxl, s_ok;
    __shared__ uint32_t s_len;
    __shared__ int s_first;
    __shared__ wave::VisitSmem<RXW, NW> sm;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool producer = warp == NW;
    Ctl *ctl = p.ctl;
    const int ntiles = p.ntx * p.nty;
    unsigned thr_maxl = 0u;
    unsigned long long visits = 0;   // producer lane 0
    uint32_t q = 0;                  // slot uses so far (same sequence on both sides)
    uint32_t pf = 0, pd = 0;         // phase bits per buffer (bit b)

    sm.zero_pad();
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&done[b], 1);
            s_fmask[b] = 0u;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t G = gridDim.x;
    if (threadIdx.x == 0) {
        s_len = ld_acquire(&ctl->list_len[0]);
        s_first = (blockIdx.x < s_len) ? take_entry(p.lists, blockIdx.x) : -1;
    }
    __syncthreads();
    if (ld_acquire(&ctl->err) & (ERR_INVAL | ERR_OBSTACLE)) return;

    wave::Visit v;
    v.g = p.g;
    v.dist_bits = 32;
    v.TY = p.TY;
    v.TXW = p.TXW;
    v.k = p.k;
    const size_t ntl = (size_t)ntiles;
    for (uint32_t s = 0;; ++s) {
        const uint32_t l0 = p.l_base + s * (uint32_t)p.k;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->work[(s + 3) % kListSlots] = 0u;
            ctl->list_len[(s + 3) % kListSlots] = 0u;
        }
        v.l0 = l0;
        v.jmax = p.k;
        if (p.max_layers && l0 + (uint32_t)p.k > p.max_layers) v.jmax = (int)(p.max_layers - l0);
        v.par = (int)(s & 1u);
        uint32_t *list = p.lists + (size_t)(s % kListSlots) * ntl;
        unsigned *work = &ctl->work[s % kListSlots];
        const uint32_t len = s_len;
        const int first = s_first;

        if (producer) {
            if (lane == 0) {
                // stage tile t (or the end marker, t < 0) into buffer b
                auto issue = [&](int t, int b) -> bool {
                    s_tile[b] = t;
                    if (t < 0) {
                        mbar_arrive(&full[b]);
                        return true;
                    }
                    const int ty = t / p.ntx, tx = t - ty * p.ntx;
                    const int gw0 = tx * p.TXW - 1, x0 = gw0 & ~3, y0 = ty * p.TY - p.k;
                    s_xoff[b] = gw0 - x0;
                    mbar_arrive_tx(&full[b], BOX_BYTES);
                    tma_load(sF[b], &tm_free, x0, y0, &full[b]);
                    return true;
                };
                auto claim = [&]() -> int {
                    if (len <= G) return -1;   // no entries past the blocks' own
                    const uint32_t i = G + atomicAdd(work, 1u);
                    return (i < len) ? take_entry(list, i) : -1;
                };
                bool ok = true;
                int t = first >= 0 ? first : claim();
                int b = (int)(q & 1u);
                ok &= issue(t, b);
                ++q;
                while (t >= 0) {
                    const int t2 = ok ? claim() : -1;
                    const int b2 = (int)(q & 1u);
                    ok &= issue(t2, b2);
                    ++q;
                    // the visit of t is done: queue what its frontier reaches
                    if (!mbar_wait(&done[b], (pd >> b) & 1u)) ok = false;
                    pd ^= 1u << b;
                    const unsigned zones = s_fmask[b];
                    s_fmask[b] = 0u;
                    const int ty = t / p.ntx, tx = t - ty * p.ntx;
                    if (zones) push_reached(p, ty, tx, zones, s + 1);
                    ++visits;
                    t = t2;
                    b = b2;
                }
                if (!ok) atomicOr(&ctl->err, ERR_TIMEOUT);
            }
        } else {
            for (;;) {
                const int b = (int)(q & 1u);
                if (threadIdx.x == 0) {
                    int t = -1;
                    if (mbar_wait(&full[b], (pf >> b) & 1u)) t = s_tile[b];
                    else atomicOr(&ctl->err, ERR_TIMEOUT);
                    s_ctile = t;
                }
                wave::bar_sync<true, NBAR>();
                const int t = s_ctile;
                // every consumer acquires the staged buffer itself (the phase
                // is complete: thread 0 saw it, so this returns at once)
                if (t >= 0) mbar_wait(&full[b], (pf >> b) & 1u);
                pf ^= 1u << b;
                ++q;
                if (t < 0) break;
                // ---- the region from the staged buffer ----
                const int w = lane % RXW;
                const int g = wave::row_group<RXW, NW>(warp, lane);
                const int r0 = g * R;
                v.ty = t / p.ntx;
                v.tx = t - v.ty * p.ntx;
                const int xo = s_xoff[b] + w;
                const bool ownW = (w >= 1) && (w <= p.TXW);
                const int gw = v.tx * p.TXW - 1 + w;
                const int y0 = v.ty * p.TY - p.k;
                uint32_t V[R], F[R], OWN[R];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int rr = r0 + i, y = y0 + rr;
                    const bool own = ownW && rr >= p.k && rr < p.k + p.TY;
                    const bool in = gw >= 0 && gw < p.g.P && y >= 0 && y < p.g.H;
                    OWN[i] = own ? 0xffffffffu : 0u;
                    F[i] = sF[b][rr * BW + xo];
                    const uint64_t vn =
                        in ? wave::ld_pair(p.g.state + 4 * ((size_t)y * p.g.P + gw) + 2 * v.par) : 0ull;
                    V[i] = (uint32_t)vn & (own ? 0xffffffffu : ~(uint32_t)(vn >> 32));
                }
                uint32_t fmask;
                unsigned lastj;
                wave::visit_core<RXW, R, NW, true>(v, sm, &ctl->err, V, F, OWN, &fmask, &lastj);
                if (fmask) atomicOr(&s_fmask[b], fmask);
                if (lastj) thr_maxl = max(thr_maxl, l0 + lastj);
                wave::bar_sync<true, NBAR>();   // all zones in
                if (threadIdx.x == 0) mbar_arrive(&done[b]);   // (TMA reads only the read-only free bits)
            }
        }

        if (!wave::grid_barrier(ctl, (s + 1) * G, p.spin_limit, &s_ok)) return;
        if (threadIdx.x == 0) {
            const uint32_t nlen = ld_acquire(&ctl->list_len[(s + 1) % kListSlots]);
            const int f = (blockIdx.x < nlen)
                              ? take_entry(p.lists + (size_t)((s + 1) % kListSlots) * ntl, blockIdx.x)
                              : -1;
            unsigned d = (nlen == 0u) || (p.max_layers && l0 + (uint32_t)p.k >= p.max_layers);
            if (!d && s + 1 >= p.sweep_cap) {
                atomicOr(&ctl->err, ERR_SWEEPS);
                d = 1;
            }
            if (d && blockIdx.x == 0) ctl->sweeps = s + 1;
            s_done = d;
            s_maxl = 0u;
            s_len = nlen;
            s_first = (blockIdx.x < nlen) ? f : -1;
        }
        __syncthreads();
        if (s_done) {
            if (thr_maxl) atomicMax(&s_maxl, thr_maxl);
            if (producer && lane == 0 && visits) atomicAdd(&ctl->visits, visits);
            __syncthreads();
            if (threadIdx.x == 0 && s_maxl) atomicMax(&ctl->max_layer, s_maxl);
            return;
        }
    }
}

// Targets: distance 0, reached bit, frontier summary of sweep 0. A target out
// of range or on an obstacle records an error and is skipped.
template <typename DT>
__global__ void k_seed(const uint32_t *targets, int n, PropParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GridDev &g = p.g;
    const uint32_t t = targets[i];
    if ((uint64_t)t >= (uint64_t)g.H * (uint64_t)g.W) {
        atomicOr(&p.ctl->err, ERR_INVAL);
        return;
    }
    const int y = (int)(t / (uint32_t)g.W), x = (int)(t % (uint32_t)g.W);
    const size_t wo = (size_t)y * g.P + (x >> 5);
    const uint32_t bit = 1u << (x & 31);
    if (!(g.free_bits[wo] & bit)) {
        atomicOr(&p.ctl->err, ERR_OBSTACLE);
        return;
    }
    reinterpret_cast<DT *>(g.dist)[t] = (DT)0;
    atomicOr(g.state + 4 * wo, bit);       // V of both pairs
    atomicOr(g.state + 4 * wo + 2, bit);
    if (p.lists) {
        const int ty = y / p.TY, tx = (x >> 5) / p.TXW;
        const int ri = y - ty * p.TY, wi = (x >> 5) - tx * p.TXW;
        push_reached(p, ty, tx, border_bits(ri, wi, bit, p.k, p.TY, p.TXW), 0u);
    }
}

// Seed from a distance plane (a run that resumes): warp per plane word, lane
// = cell. A cell at distance <= from is reached and keeps its distance (an
// obstacle marked reached is ERR_INVAL); every other cell starts unreached.
// Tiles holding cells at distance `from` are queued for sweep 0 with the
// border zones those frontier cells touch.
template <typename DT>
__global__ void k_seed_plane(const DT *__restrict__ din, PropParams p) {
    const GridDev &g = p.g;
    const size_t wid = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= (size_t)g.H * g.P) return;   // whole warp leaves together
    const int y = (int)(wid / (size_t)g.P), w = (int)(wid % (size_t)g.P);
    const int x = 32 * w + lane;
    const DT INF = (DT)~(DT)0;
    const uint32_t from = p.l_base;
    DT d = INF;
    if (x < g.W) d = din[(size_t)y * g.W + x];
    const bool reached = x < g.W && d != INF && (uint32_t)d <= from;
    const unsigned vb = __ballot_sync(0xffffffffu, reached);
    const unsigned fb = __ballot_sync(0xffffffffu, reached && (uint32_t)d == from);
    if (x < g.W) reinterpret_cast<DT *>(g.dist)[(size_t)y * g.W + x] = reached ? d : INF;
    if (lane == 0) {
        const size_t wo = (size_t)y * g.P + w;
        if (vb & ~g.free_bits[wo]) atomicOr(&p.ctl->err, ERR_INVAL);
        const uint32_t v = vb & g.free_bits[wo];
        wave::st_pair(g.state + 4 * wo, v, 0u);
        wave::st_pair(g.state + 4 * wo + 2, v, 0u);
        const uint32_t f = fb & v;
        if (f && w < p.ntx * p.TXW) {
            const int ty = y / p.TY, tx = w / p.TXW;
            push_reached(p, ty, tx, border_bits(y - ty * p.TY, w - tx * p.TXW, f, p.k, p.TY, p.TXW), 0u);
        }
    }
}

// One layer of the recursive mode on the distance plane: an unreached free
// cell with a neighbour at distance layer - 1 gets distance layer.
template <typename DT>
__global__ void k_plain_layer(GridDev g, uint32_t layer, Ctl *ctl) {
    const DT INF = (DT)~(DT)0;
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    DT *distw = reinterpret_cast<DT *>(g.dist);
    const DT want = (DT)(layer - 1u);
    const size_t n = (size_t)g.H * g.W;
    bool any = false;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        if (dist[c] != INF) continue;
        const int y = (int)(c / g.W), x = (int)(c % g.W);
        if (!((g.free_bits[(size_t)y * g.P + (x >> 5)] >> (x & 31)) & 1u)) continue;
        bool hit = false;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = y + dy, xx = x + dx;
                if ((dy || dx) && yy >= 0 && xx >= 0 && yy < g.H && xx < g.W &&
                    dist[(size_t)yy * g.W + xx] == want)
                    hit = true;
            }
        if (hit) {
            if (sizeof(DT) == 2 && layer > 0xfffeu) {
                atomicOr(&ctl->err, ERR_OVERFLOW);
            } else {
                distw[c] = (DT)layer;
                any = true;
            }
        }
    }
    const unsigned who = __ballot_sync(0xffffffffu, any);
    if (who && (threadIdx.x & 31) == __ffs(who) - 1) atomicMax(&ctl->plain_last, layer);
}

template <int RXW, int R, int NW, int MINB, int WPL = 1>
void *variant_ptr(bool u16) {
    return u16 ? (void *)k_propagate<RXW, R, NW, MINB, uint16_t, WPL>
               : (void *)k_propagate<RXW, R, NW, MINB, uint32_t, WPL>;
}

// Compiled tile shapes: {region words, rows per lane, warps per block, blocks
// per SM the register budget aims at}. Region rows = warps * (32 / words) *
// rows per lane; interior = region minus k rows top and bottom and one word
// left and right.
constexpr VariantDesc kVariants[] = {
    {8, 4, 8, 3, 0},    // 128 rows x 256 cells
    {8, 8, 8, 2, 0},    // 256 rows x 256 cells
    {16, 4, 8, 3, 0},   //  64 rows x 512 cells
    {4, 8, 8, 2, 0},    // 512 rows x 128 cells
    {8, 4, 4, 5, 0},    //  64 rows x 256 cells
    {16, 8, 8, 2, 0},   // 128 rows x 512 cells
    {8, 4, 8, 2, 1},    // 128 rows x 256 cells, TMA-staged, + producer warp (uint32 planes)
    {8, 2, 16, 2, 0},   // 128 rows x 256 cells, 2 rows per lane (shorter per-layer chains)
    {8, 1, 32, 1, 0},   // 128 rows x 256 cells, 1 row per lane, 1024 threads
    {8, 2, 8, 3, 0, 2},   // 128 rows x 256 cells, 2 words x 2 rows per lane
    {8, 4, 8, 2, 0, 2},   // 256 rows x 256 cells, 2 words x 4 rows per lane
    {8, 8, 4, 4, 0},    // 128 rows x 256 cells, 4 warps of 8 rows per lane (fewer warps per barrier)
    {8, 4, 4, 4, 0, 2},   // 128 rows x 256 cells, 4 warps of 2 words x 4 rows per lane
    {8, 4, 3, 5, 0, 2},   //  96 rows x 256 cells, 3 warps of 2 words x 4 rows per lane
};

void *variant_fn(int v, int dist_bits) {
    const bool u16 = dist_bits == 16;
    switch (v) {
        case 0: return variant_ptr<8, 4, 8, 3>(u16);
        case 1: return variant_ptr<8, 8, 8, 2>(u16);
        case 2: return variant_ptr<16, 4, 8, 3>(u16);
        case 3: return variant_ptr<4, 8, 8, 2>(u16);
        case 4: return variant_ptr<8, 4, 4, 5>(u16);
        case 5: return variant_ptr<16, 8, 8, 2>(u16);
        case 6: return u16 ? nullptr : (void *)k_propagate_tma<8, 4, 8>;
        case 7: return variant_ptr<8, 2, 16, 2>(u16);
        case 8: return variant_ptr<8, 1, 32, 1>(u16);
        case 9: return variant_ptr<8, 2, 8, 3, 2>(u16);
        case 10: return variant_ptr<8, 4, 8, 2, 2>(u16);
        case 11: return variant_ptr<8, 8, 4, 4>(u16);
        case 12: return variant_ptr<8, 4, 4, 4, 2>(u16);
        case 13: return variant_ptr<8, 4, 3, 5, 2>(u16);
        default: return nullptr;
    }
}

}  // namespace

int num_variants() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }

VariantDesc variant_desc(int v) { return kVariants[v]; }

int variant_threads(int v) { return (kVariants[v].nwarps + kVariants[v].tma) * 32; }

cudaError_t propagate_blocks_per_sm(int v, int dist_bits, int *out) {
    void *fn = variant_fn(v, dist_bits);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, variant_threads(v), 0);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
        else
            cudaGetLastError();
    });
    return fn;
}

// A bit plane (H rows x P uint32 words, P a multiple of 4) as a 2-D tensor
// with a box of bw words x ry rows; out-of-range elements read as zero.
cudaError_t plane_map(CUtensorMap *m, const void *base, int P, int H, int bw, int ry) {
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)H};
    cuuint64_t strides[1] = {(cuuint64_t)P * 4u};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)ry};
    cuuint32_t es[2] = {1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_propagate(int v, int dist_bits, const PropParams &p, int blocks,
                             cudaStream_t st) {
    void *fn = variant_fn(v, dist_bits);
    if (!fn) return cudaErrorInvalidValue;
    PropParams pp = p;
    count_launch();
    if (!kVariants[v].tma) {
        void *args[] = {&pp};
        return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(variant_threads(v)), args, 0, st);
    }
    const VariantDesc &d = kVariants[v];
    const int ry = region_rows(d), bw = (d.rxw + 6) / 4 * 4;
    CUtensorMap mf;
    cudaError_t e = plane_map(&mf, p.g.free_bits, p.g.P, p.g.H, bw, ry);
    if (e != cudaSuccess) return e;
    void *args[] = {&mf, &pp};
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(variant_threads(v)), args, 0, st);
}

template <int TXW>
static cudaError_t launch_decode_txw(const PropParams &p, int dist_bits, int sm_count, uint32_t slots,
                                     cudaStream_t st) {
    // a band of at most 36 KB with 16-bit layer codes (a whole 80-row
    // interior for the usual tile shapes, so each log entry is read once, and
    // six blocks per SM), plus its reached and covered words
    int band = (36 * 1024) / (TXW * (34 * 2 + 8));
    band = band < 1 ? 1 : (band > p.TY ? p.TY : band);
    const size_t smem = decode_band_words(band, TXW) * sizeof(uint32_t);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        // the largest shared-memory carveout, so that six blocks fit per SM
        const void *fns[2] = {(const void *)k_log_decode<uint16_t, TXW>, (const void *)k_log_decode<uint32_t, TXW>};
        for (const void *f : fns) {
            if (attr == cudaSuccess)
                attr = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 * 1024);
            if (attr == cudaSuccess)
                attr = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                            cudaSharedmemCarveoutMaxShared);
        }
    });
    if (attr != cudaSuccess) return attr;
    const int ntiles = p.ntx * p.nty;
    const int most = sm_count * 6;
    const int blocks = ntiles < most ? ntiles : most;
    count_launch();
    if (dist_bits == 16)
        k_log_decode<uint16_t, TXW><<<blocks, 256, smem, st>>>(p, band, slots);
    else
        k_log_decode<uint32_t, TXW><<<blocks, 256, smem, st>>>(p, band, slots);
    return cudaGetLastError();
}

cudaError_t launch_log_decode(const PropParams &p, int dist_bits, int sm_count, uint32_t slots,
                              cudaStream_t st) {
    if (!p.log) return cudaSuccess;
    if (slots < 1 || slots > kTileSlots) slots = kTileSlots;
    switch (p.TXW) {   // interior words of a tile: region words (4, 8 or 16) - 2
        case 2: return launch_decode_txw<2>(p, dist_bits, sm_count, slots, st);
        case 6: return launch_decode_txw<6>(p, dist_bits, sm_count, slots, st);
        case 14: return launch_decode_txw<14>(p, dist_bits, sm_count, slots, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_seed(const uint32_t *targets, int n, const PropParams &p, int dist_bits,
                        cudaStream_t st) {
    const int tb = 256, nb = (n + tb - 1) / tb;
    count_launch();
    if (dist_bits == 16) k_seed<uint16_t><<<nb, tb, 0, st>>>(targets, n, p);
    else k_seed<uint32_t><<<nb, tb, 0, st>>>(targets, n, p);
    return cudaGetLastError();
}

cudaError_t launch_seed_plane(const void *din, const PropParams &p, int dist_bits, cudaStream_t st) {
    const size_t words = (size_t)p.g.H * p.g.P;
    const int wpb = 8;
    const size_t nb = (words + wpb - 1) / wpb;
    count_launch();
    if (dist_bits == 16) k_seed_plane<uint16_t><<<(unsigned)nb, wpb * 32, 0, st>>>((const uint16_t *)din, p);
    else k_seed_plane<uint32_t><<<(unsigned)nb, wpb * 32, 0, st>>>((const uint32_t *)din, p);
    return cudaGetLastError();
}

cudaError_t launch_plain_seed(const uint32_t *targets, int n, const GridDev &g, int dist_bits,
                              Ctl *ctl, cudaStream_t st) {
    PropParams p{};
    p.g = g;
    p.ctl = ctl;
    p.lists = nullptr;
    return launch_seed(targets, n, p, dist_bits, st);
}

cudaError_t launch_plain_layer(const GridDev &g, int dist_bits, uint32_t layer, Ctl *ctl,
                               cudaStream_t st) {
    const size_t n = (size_t)g.H * g.W;
    const int tb = 256;
    const size_t want = (n + tb - 1) / tb;
    const int nb = (int)(want < 152 * 64 ? want : 152 * 64);
    count_launch();
    if (dist_bits == 16) k_plain_layer<uint16_t><<<nb, tb, 0, st>>>(g, layer, ctl);
    else k_plain_layer<uint32_t><<<nb, tb, 0, st>>>(g, layer, ctl);
    return cudaGetLastError();
}

}  // namespace mpn
