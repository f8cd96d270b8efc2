// Device code shared by the single-grid and the batched propagation kernels:
// memory-order helpers, the bounded grid barrier, and one tile visit (k layers
// of the max-pool wave on bit planes in registers).
//
// One layer of the paper maps A_{l-1} to ReLU(maxpool3x3(A_{l-1}) + I_e + I_s)
// (Methods, "Activity Map Generation"). Only whether a cell is positive
// matters for its first-activation layer, and the positive set of A_l is the
// 3x3 dilation of the positive set of A_{l-1} intersected with the free cells
// (an obstacle's -maxint keeps it at zero; a source stays positive). So on a
// 1-bit-per-cell plane a layer is
//     reached_l = reached_{l-1} | (dilate3x3(reached_{l-1}) & free),
// and the cells new at layer l get distance l. A 32-bit word holds 32 cells of
// a row: one layer costs a few funnel shifts and three-input logic operations
// per word instead of nine max operations per cell.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "mpn_internal.cuh"

namespace mpn {
namespace wave {

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A {V, Np} pair of the propagation state as one 64-bit access (V in the low
// word).
__device__ __forceinline__ uint64_t ld_pair(const uint32_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_pair(uint32_t *p, uint32_t v, uint32_t n) {
    const uint64_t x = (uint64_t)v | ((uint64_t)n << 32);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(x) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a co-resident (cooperative) grid on a monotonic
// arrival counter: the n-th barrier of a launch completes when the counter
// reaches target = n * blocks, so no block resets or bumps anything after
// arriving. The wait is bounded: past spin_limit polls the block records
// ERR_TIMEOUT and returns false; a block that sees ERR_TIMEOUT already recorded
// also stops waiting, so one expired wait ends every block instead of starting
// a new wait in each.
__device__ __forceinline__ bool grid_barrier(Ctl *c, unsigned target, unsigned spin_limit,
                                             unsigned *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        // arrive with release semantics (the block's writes, ordered before
        // this thread by the block barrier, become visible with it) and wait
        // with acquire loads: no separate fences
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&c->bar_count) : "memory");
        unsigned ok = 1, spins = 0;
        while (ld_acquire(&c->bar_count) < target) {
            ++spins;
            if ((spins & 63u) == 0u && (ld_acquire(&c->err) & ERR_TIMEOUT)) {   // another block gave up
                ok = 0;
                break;
            }
            if (spins > spin_limit) {
                atomicOr(&c->err, ERR_TIMEOUT);
                ok = 0;
                break;
            }
            if (spins > 8) __nanosleep(32);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Rank of this block for the fixed one-entry-per-block deal of a tile list
// (entry r goes to the block of rank r without an atomic). The hardware puts
// consecutive block indices on the same SM (on a GB300, blocks 0..11 of a
// three-per-SM grid share four SMs), so a short list dealt by block index
// would run several visits on one SM while most SMs idle. Ranked by the
// block's place among the blocks of its SM first, the first block of every
// SM comes before any second one. Thread 0 of every block of the grid calls
// it once, at the start; cnt holds kRankWords counters that are zero at the
// launch (256 per SM, 32 per place, one barrier). The ranks are a permutation
// of 0 .. gridDim.x - 1. A wait past spin_limit records ERR_TIMEOUT in *err
// and returns -1; without counters (cnt null) the rank is the block index.
__device__ __forceinline__ int block_rank(uint32_t *cnt, unsigned spin_limit, uint32_t *err) {
    if (!cnt) return (int)blockIdx.x;
    unsigned nsm, sid;
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsm));
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sid));
    if (nsm > 256u) return (int)blockIdx.x;   // (the same for every block)
    const unsigned place = atomicAdd(cnt + sid, 1u);   // < 32 resident blocks per SM
    const unsigned pos = atomicAdd(cnt + 256 + place, 1u);
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt + 288) : "memory");
    unsigned spins = 0;
    while (ld_acquire(cnt + 288) < gridDim.x) {
        if (++spins > spin_limit || ((spins & 63u) == 0u && (ld_acquire(err) & ERR_TIMEOUT))) {
            atomicOr(err, ERR_TIMEOUT);
            return -1;
        }
        if (spins > 8) __nanosleep(32);
    }
    unsigned base = 0;
    for (unsigned j = 0; j < place; ++j) base += ld_relaxed(cnt + 256 + j);
    return (int)(base + pos);
}

// 3x3 dilation along the row: v | v shifted one cell left | one cell right,
// with the carries from the neighbouring words of the same row (the lanes of
// one row group hold consecutive words). At the region's outer words the
// shuffle returns the lane's own word, so the outermost cell of the region can
// pick up a wrong bit; that error moves one cell per layer and, with a one-word
// (32-cell) horizontal halo and at most 32 layers per visit, never reaches the
// interior.
template <int RXW>
__device__ __forceinline__ uint32_t hdil(uint32_t v) {
    const uint32_t left = __shfl_up_sync(0xffffffffu, v, 1, RXW);
    const uint32_t right = __shfl_down_sync(0xffffffffu, v, 1, RXW);
    return v | __funnelshift_l(left, v, 1) | __funnelshift_r(v, right, 1);
}

// Which border zones of the tile interior a set of frontier cells touches.
// ri: interior row, wi: interior word, bits: frontier cells of that word.
__device__ __forceinline__ uint32_t border_bits(int ri, int wi, uint32_t bits, int k, int TY,
                                                int TXW) {
    if (!bits) return 0u;
    const uint32_t lowk = (k >= 32) ? 0xffffffffu : ((1u << k) - 1u);
    const uint32_t highk = (k >= 32) ? 0xffffffffu : ~((1u << (32 - k)) - 1u);
    const bool top = ri < k, bot = ri >= TY - k;
    const bool left = (wi == 0) && (bits & lowk);
    const bool right = (wi == TXW - 1) && (bits & highk);
    uint32_t m = FB_ANY;
    if (top) m |= FB_N;
    if (bot) m |= FB_S;
    if (left) m |= FB_W;
    if (right) m |= FB_E;
    if (top && left) m |= FB_NW;
    if (top && right) m |= FB_NE;
    if (bot && left) m |= FB_SW;
    if (bot && right) m |= FB_SE;
    return m;
}

// Block-level OR-reduction barrier: all threads of the block (NAMED false) or
// only the NBAR consumer threads on named barrier 1 (NAMED true), so that a
// producer warp can run on without joining the per-layer barriers.
template <bool NAMED, int NBAR>
__device__ __forceinline__ int bar_or(int pred) {
    if (!NAMED) return __syncthreads_or(pred);
    uint32_t out;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(out) : "r"((uint32_t)pred), "n"(NBAR) : "memory");
    return (int)out;
}

template <bool NAMED, int NBAR>
__device__ __forceinline__ void bar_sync() {
    if (!NAMED) {
        __syncthreads();
        return;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(NBAR) : "memory");
}

// A callback that visit_core runs once, on every thread, a few layers into
// the visit (after the first four layers, or at the end of a shorter visit):
// a point at which the block's earlier memory operations have completed.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// One tile visit's inputs.
struct Visit {
    GridDev g;            // planes of the grid the tile belongs to
    int par;              // parity of the sweep: the visit reads {V, Npar}
    int dist_bits;        // 16 or 32
    int TY, TXW, k;       // tile geometry and depth
    int ty, tx;           // tile coordinates within its grid
    uint32_t l0;          // layer at the start of the sweep
    int jmax;             // layers to run (k, or fewer at a layer cap)
};

// Row group of a lane. The NW * 32 / RXW row groups of a region (R rows
// each, top to bottom) are dealt to the warps round-robin: group g sits in warp
// g % NW, lane group g / NW. So every warp holds rows of the top halo, the
// interior and the bottom halo alike, and the per-warp distance write-out at
// the end of a visit (one store per reached word) is balanced.
template <int RXW, int NW>
__device__ __forceinline__ int row_group(int warp, int lane) {
    return (lane / RXW) * NW + warp;
}

// Shared-memory slot of word w of row group g in the halo exchange: the slots
// of a warp are 32 consecutive words, so the writes and the reads of the
// neighbouring groups' rows are free of bank conflicts.
template <int RXW, int NW>
__device__ __forceinline__ int xslot(int g, int w) {
    return (g % NW) * 32 + (g / NW) * RXW + w;
}

// Where a visit leaves its activation records: chunk *s_chunk of the
// activation log, with *s_cursor entries already used (both in shared memory,
// set by the block before the visit's first barrier; the block has reserved
// the visit's header entry in front of them). No log, or *s_chunk < 0: the
// visit writes its distances itself.
struct LogSink {
    uint32_t *log = nullptr;
    const int *s_chunk = nullptr;
    unsigned *s_cursor = nullptr;
};

template <int RXW, int NW, int WPL = 1>
struct VisitSmem {
    // per layer parity: top row of each group, dilated along the row (WPL
    // words per lane); past the NW * 32 lanes' slots: zero, the region's outer
    // neighbours
    uint32_t xtop[2][(NW * 32 + 1) * WPL];
    uint32_t xbot[2][(NW * 32 + 1) * WPL];   // bottom row
    __device__ __forceinline__ void zero_pad() {
        if (threadIdx.x < 4 * WPL) {
            const int q = threadIdx.x / WPL, u = threadIdx.x % WPL;
            (q < 2 ? xtop : xbot)[q & 1][NW * 32 * WPL + u] = 0u;
        }
    }
};

// 3x3 dilation along the row for a lane holding two adjacent words (a, b) of
// a row: the carries into a come from the left lane's b and into b from the
// right lane's a. Same edge argument as hdil.
template <int LG>
__device__ __forceinline__ void hdil2(uint32_t a, uint32_t b, uint32_t &ha, uint32_t &hb) {
    const uint32_t left = __shfl_up_sync(0xffffffffu, b, 1, LG);
    const uint32_t right = __shfl_down_sync(0xffffffffu, a, 1, LG);
    ha = a | __funnelshift_l(left, a, 1) | __funnelshift_r(a, b, 1);
    hb = b | __funnelshift_l(a, b, 1) | __funnelshift_r(b, right, 1);
}

// Advance one tile by up to v.jmax layers from its region already in
// registers (V: visit bits as of the start of the sweep, F: free bits, OWN:
// all-ones on this tile's interior words), write the distances of the cells it
// reaches (a uint16 overflow sets ERR_OVERFLOW in *err), publish its new visit
// bits (after the this-sweep bits) and return the border zones of its frontier
// (cells reached at layer l0 + k) and, per thread, the last layer at which one
// of this thread's cells was reached. Every participating thread calls it; it
// contains barriers (block-wide, or named barrier 1 when NAMED).
//
// Block layout: a row group is RXW / WPL consecutive lanes holding RXW
// consecutive words of R consecutive rows (WPL adjacent words per lane per
// row, in registers; slot s = i * WPL + u is word u of row i). Region =
// (NW * 32 / (RXW / WPL) * R) rows x RXW words; interior = rows [k, RY - k)
// x words [1, RXW - 1).
template <int RXW, int R, int NW, bool NAMED, int WPL = 1, typename Hook = NoHook>
__device__ __forceinline__ void visit_core(const Visit &v, VisitSmem<RXW, NW, WPL> &sm, uint32_t *err,
                                           uint32_t (&V)[R * WPL], const uint32_t (&F)[R * WPL],
                                           const uint32_t (&OWN)[R * WPL], uint32_t *fmask_out,
                                           unsigned *lastj_out, const LogSink &lg = LogSink(),
                                           unsigned *jrun_out = nullptr, const Hook &hook = Hook()) {
    static_assert(WPL == 1 || WPL == 2, "words per lane");
    constexpr int LG = RXW / WPL;   // lanes per row group
    constexpr int GPW = 32 / LG;
    constexpr int G = NW * GPW;
    constexpr int S = R * WPL;      // words per thread
    constexpr int NBAR = NW * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wl = lane % LG;        // lane within the row group
    const int g = row_group<LG, NW>(warp, lane);
    const int r0 = g * R;
    const int k = v.k, TY = v.TY, TXW = v.TXW;
    const GridDev &gd = v.g;
    const int y0 = v.ty * TY - k;
    const int gw0 = v.tx * TXW - 1 + wl * WPL;   // word u of a row is gw0 + u
    const int slot = (warp * 32 + lane) * WPL;   // == xslot(g, wl) * WPL
    const int slot_up = (g > 0 ? xslot<LG, NW>(g - 1, wl) : NW * 32) * WPL;
    const int slot_dn = (g < G - 1 ? xslot<LG, NW>(g + 1, wl) : NW * 32) * WPL;
    uint32_t V0[S];   // visit bits at the start of the visit
#pragma unroll
    for (int s = 0; s < S; ++s) V0[s] = V[s];

    // ---- up to k layers in registers ----
    // Activation times as a bit-sliced Gray-code counter: P[b][s] holds bit b
    // of gray(t), t = layer - l0 - 1. Every cell not reached yet carries the
    // same count, gray(j - 1) before layer j, so advancing all of them to
    // gray(j) flips the single plane ctz(j) on the unreached cells (one
    // operation per word and layer); a cell keeps its value once reached, and
    // each cell's distance is written once, at the end of the visit.
    uint32_t P[5][S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int b = 0; b < 5; ++b) P[b][s] = 0u;
    }
    // Per layer: every row dilated along the row first (the shuffles of the
    // inner rows overlap the wait at the barrier), the group's top and bottom
    // rows exchanged through shared memory, then a row's new bits are the
    // vertical OR of three dilated rows within the free cells. The bits a
    // visit reaches are recovered at the end against V0. Layers run in
    // fours (j = 1, 2, 3, 0 mod 4), so the Gray plane of three of them is
    // known at compile time; a layer j = 0 mod 4 records whether it changed
    // anything and the next layer's barrier ORs that over the block and ends
    // the visit if nothing did (a stable region costs at most three extra
    // layers). The row groups at the region's top and bottom edge read a
    // zero exchange slot.
    uint32_t changed = 1u;
    unsigned lastj = 0u;
    // one layer with the exchange slots of its parity; false: region stable.
    // kind (compile time): check the stability flag, record it, or neither.
    using Check = std::integral_constant<int, 1>;
    using Record = std::integral_constant<int, 0>;
    using Plain = std::integral_constant<int, 2>;
    auto layer = [&](uint32_t *xt, uint32_t *xb, auto kind) -> bool {
        uint32_t h[S];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (WPL == 1) h[i] = hdil<LG>(V[i]);
            else hdil2<LG>(V[i * WPL], V[i * WPL + WPL - 1], h[i * WPL], h[i * WPL + WPL - 1]);
        }
#pragma unroll
        for (int u = 0; u < WPL; ++u) {
            xt[slot + u] = h[u];
            xb[slot + u] = h[(R - 1) * WPL + u];
        }
        if (decltype(kind)::value == Check::value) {
            if (!bar_or<NAMED, NBAR>(changed != 0u)) return false;
        } else {
            bar_sync<NAMED, NBAR>();
        }
        uint32_t hUp[WPL], hDn[WPL];
#pragma unroll
        for (int u = 0; u < WPL; ++u) {
            hUp[u] = xb[slot_up + u];
            hDn[u] = xt[slot_dn + u];
        }
        if (decltype(kind)::value == Record::value) changed = 0u;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int i = s / WPL, u = s % WPL;
            const uint32_t up = (i > 0) ? h[s - WPL] : hUp[u];
            const uint32_t dn = (i < R - 1) ? h[s + WPL] : hDn[u];
            const uint32_t vn = V[s] | ((up | h[s] | dn) & F[s]);
            if (decltype(kind)::value == Record::value) changed |= vn ^ V[s];
            V[s] = vn;
        }
        return true;
    };
    // unreached cells: gray(j - 1) -> gray(j), plane ctz(j)
#define MPN_FLIP(B) _Pragma("unroll") for (int s = 0; s < S; ++s) P[B][s] ^= ~V[s]
    int jdone = v.jmax;   // layers run (fewer when the region turns stable)
    bool hooked = false;
    for (int j = 1; j <= v.jmax; j += 4) {   // j = 1 mod 4
        if (j == 5) {
            hook();
            hooked = true;
        }
        if (!layer(sm.xtop[1], sm.xbot[1], Check())) {
            jdone = j - 1;
            break;
        }
        if (j == v.jmax) break;
        MPN_FLIP(0);
        if (!layer(sm.xtop[0], sm.xbot[0], Plain())) break;
        if (j + 1 == v.jmax) break;
        MPN_FLIP(1);
        if (!layer(sm.xtop[1], sm.xbot[1], Plain())) break;
        if (j + 2 == v.jmax) break;
        MPN_FLIP(0);
        if (!layer(sm.xtop[0], sm.xbot[0], Record())) break;
        if (j + 3 == v.jmax) break;
        switch (__ffs(j + 3) - 1) {   // 2..4 (j + 3 < 32), block-uniform
            case 2: MPN_FLIP(2); break;
            case 3: MPN_FLIP(3); break;
            default: MPN_FLIP(4); break;
        }
    }
#undef MPN_FLIP
    if (!hooked) hook();
    if (jrun_out) *jrun_out = (unsigned)jdone;

    // cells of this tile's interior first reached in this visit
    uint32_t NB[S];
#pragma unroll
    for (int s = 0; s < S; ++s) NB[s] = (V[s] ^ V0[s]) & OWN[s];

    // ---- the last layer at which one of this thread's cells was reached ----
    // (a bit-sliced maximum of t over the reached cells, from the planes
    // turned from Gray code into binary, most significant bit first). Only
    // when the visit writes its distances itself: with the activation log the
    // decode sees every cell's layer and takes the maximum there.
    const int chunk = lg.log ? *lg.s_chunk : -1;   // block-uniform
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (chunk >= 0 || !NB[s]) continue;
        uint32_t B[5];
        B[4] = P[4][s];
#pragma unroll
        for (int b = 3; b >= 0; --b) B[b] = P[b][s] ^ B[b + 1];
        uint32_t cand = NB[s], m = 0u;
#pragma unroll
        for (int b = 4; b >= 0; --b) {
            const uint32_t hit = cand & B[b];
            if (hit) {
                m |= 1u << b;
                cand = hit;
            }
        }
        lastj = max(lastj, m + 1u);
    }

    // ---- frontier zones: cells reached at layer l0 + k ----
    uint32_t fmask = 0u;
    if (v.jmax == k) {
        const uint32_t gk = (uint32_t)(k - 1) ^ ((uint32_t)(k - 1) >> 1);   // gray(k - 1)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            uint32_t last = NB[s];
#pragma unroll
            for (int b = 0; b < 5; ++b) last &= ((gk >> b) & 1) ? P[b][s] : ~P[b][s];
            fmask |= border_bits(r0 + s / WPL - k, wl * WPL + s % WPL - 1, last, k, TY, TXW);
        }
    }
    *fmask_out = fmask;
    *lastj_out = lastj;

    // ---- distances of the cells first reached in this visit ----
    if (chunk >= 0) {
        // one activation-log entry per changed word: the warp reserves its
        // entries with one shared-memory atomic and writes each as two 16-byte
        // stores (the warp's entries are consecutive)
        const uint32_t cbase = (uint32_t)chunk * kLogChunk;
        unsigned act[S];
        uint32_t tot = 0u;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            act[s] = __ballot_sync(0xffffffffu, NB[s] != 0u);
            tot += (uint32_t)__popc(act[s]);
        }
        uint32_t at = 0u;
        if (lane == 0 && tot) at = atomicAdd(lg.s_cursor, tot);
        at = __shfl_sync(0xffffffffu, at, 0);
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (NB[s]) {
                const uint32_t idx = cbase + at + (uint32_t)__popc(act[s] & below);
                uint4 *e = reinterpret_cast<uint4 *>(lg.log + (size_t)idx * kLogFields);
                // the word's place in the tile interior: row * TXW + word
                const uint32_t pos = (uint32_t)(r0 + s / WPL - k) * (uint32_t)TXW +
                                     (uint32_t)(wl * WPL + s % WPL - 1);
                e[0] = make_uint4(pos, NB[s], P[0][s], P[1][s]);
                e[1] = make_uint4(P[2][s], P[3][s], P[4][s], 0u);
            }
            at += (uint32_t)__popc(act[s]);
        }
    } else {
    // The warp writes one changed word at a time: 32 lanes, 32 consecutive
    // cells, one coalesced store.
#pragma unroll
    for (int s = 0; s < S; ++s) {
        unsigned act = __ballot_sync(0xffffffffu, NB[s] != 0u);
        while (act) {
            const int src = __ffs(act) - 1;
            act &= act - 1u;
            const uint32_t nb = __shfl_sync(0xffffffffu, NB[s], src);
            uint32_t off = 0u;   // gray(t) of this lane's cell, then t
#pragma unroll
            for (int b = 0; b < 5; ++b)
                off |= ((__shfl_sync(0xffffffffu, P[b][s], src) >> lane) & 1u) << b;
            off ^= off >> 1;
            off ^= off >> 2;
            off ^= off >> 4;
            const int sw = (src % LG) * WPL + s % WPL;       // source word column
            const int sg = row_group<LG, NW>(warp, src);     // source row group
            const int y = y0 + sg * R + s / WPL;
            const size_t cell = (size_t)y * gd.W + (size_t)(v.tx * TXW - 1 + sw) * 32 + lane;
            if ((nb >> lane) & 1u) {
                const uint32_t layer = v.l0 + 1u + off;
                if (v.dist_bits == 16) {
                    if (layer > 0xfffeu) atomicOr(err, ERR_OVERFLOW);
                    else reinterpret_cast<uint16_t *>(gd.dist)[cell] = (uint16_t)layer;
                } else {
                    reinterpret_cast<uint32_t *>(gd.dist)[cell] = layer;
                }
            }
        }
    }

    }   // log or direct

    // ---- publish: {V, this sweep's new bits} for this parity, {V, 0} for
    // the other (a later sweep of that parity sees no stale bits of this word)
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (!NB[s]) continue;
        uint32_t *st = gd.state + 4 * ((size_t)(y0 + r0 + s / WPL) * gd.P + gw0 + s % WPL);
        st_pair(st + 2 * v.par, V[s], NB[s]);
        st_pair(st + 2 * (v.par ^ 1), V[s], 0u);
    }
}

// A tile visit that loads its own region from global memory (the
// register-only kernels). Halo words of other tiles are read as of the start
// of the sweep: the {V, Npar} pair comes in one load, and a word that its
// owner changed in this sweep has exactly the bits new in this sweep in Npar.
// (A word last changed two or more sweeps back may still carry that sweep's
// bits in Npar; those cells' whole neighbourhoods were reached by then, so
// hiding them changes nothing inside the tile.)
template <int RXW, int R, int NW, int WPL = 1, typename Hook = NoHook>
__device__ __forceinline__ void visit_tile(const Visit &v, VisitSmem<RXW, NW, WPL> &sm, uint32_t *err,
                                           uint32_t *fmask_out, unsigned *lastj_out,
                                           const LogSink &lg = LogSink(),
                                           unsigned *jrun_out = nullptr, const Hook &hook = Hook()) {
    constexpr int LG = RXW / WPL;
    constexpr int S = R * WPL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wl = lane % LG;
    const int g = row_group<LG, NW>(warp, lane);
    const int r0 = g * R;
    const int k = v.k, TY = v.TY, TXW = v.TXW;
    const GridDev &gd = v.g;
    const int y0 = v.ty * TY - k;
    const int gw0 = v.tx * TXW - 1 + wl * WPL;
    uint32_t V[S], F[S], OWN[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int rr = r0 + s / WPL, y = y0 + rr;
        const int w = wl * WPL + s % WPL, gw = gw0 + s % WPL;
        const bool in = gw >= 0 && gw < gd.P && y >= 0 && y < gd.H;
        const bool own = w >= 1 && w <= TXW && rr >= k && rr < k + TY;
        const size_t off = (size_t)y * gd.P + gw;
        OWN[s] = own ? 0xffffffffu : 0u;
        F[s] = in ? __ldg(gd.free_bits + off) : 0u;
        const uint64_t vn = in ? ld_pair(gd.state + 4 * off + 2 * v.par) : 0ull;
        V[s] = (uint32_t)vn & (own ? 0xffffffffu : ~(uint32_t)(vn >> 32));
    }
    visit_core<RXW, R, NW, false, WPL>(v, sm, err, V, F, OWN, fmask_out, lastj_out, lg, jrun_out, hook);
}

}  // namespace wave
}  // namespace mpn
