// Activity propagation: the stack of max-pool layers (Methods, "Activity Map
// Generation", Fig. 1) computed on bit planes.
//
// One layer of the paper maps A_{l-1} to ReLU(maxpool3x3(A_{l-1}) + I_e + I_s).
// Only whether a cell is positive matters for its first-activation layer, and
// the positive set of A_l is the 3x3 dilation of the positive set of A_{l-1},
// intersected with the free cells (an obstacle's -maxint keeps it at zero;
// a source stays positive). So a layer is, on a 1-bit-per-cell plane,
//     reached_l = reached_{l-1} | (dilate3x3(reached_{l-1}) & free),
// and the cells new at layer l get distance l. A 32-bit word holds 32 cells of
// a row, so one layer is a handful of funnel shifts and three-input logic ops
// per word instead of nine max operations per cell.
//
// k_propagate is persistent and temporally blocked: the grid is cut into tiles;
// a tile visit loads the tile plus a halo of k rows and one word (32 cells) on
// each side into registers and advances k layers there, then writes back the
// interior. Sweeps of k layers are separated by a grid-wide barrier; inside a
// sweep only tiles that the frontier can reach within k layers are visited:
// a visit that ends with frontier cells queues the tiles they can reach for
// the next sweep, and blocks claim work from that list.
// Halo cells are read as of the start of the sweep: a neighbour tile already
// advanced in this sweep has also published which of its cells it reached in
// this sweep (nb plane of the sweep's parity), and those bits are masked out.
//
// k_plain_layer is the paper's recursive mode, one launch per layer over the
// whole distance plane, kept as the baseline.
#include <cuda_runtime.h>

#include "mpn_internal.cuh"

namespace mpn {

namespace {

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a co-resident (cooperative) grid. The wait is bounded:
// past spin_limit polls the block records ERR_TIMEOUT and returns false; a
// block that sees ERR_TIMEOUT already recorded also stops waiting, so one
// expired wait ends every block instead of starting a new wait in each.
__device__ bool grid_barrier(Ctl *c, unsigned nblocks, unsigned spin_limit) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ok = 1;
        const unsigned gen = ld_acquire(&c->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            unsigned spins = 0;
            while (ld_acquire(&c->bar_gen) == gen) {
                if (ld_acquire(&c->err) & ERR_TIMEOUT) {   // another block gave up
                    ok = 0;
                    break;
                }
                if (++spins > spin_limit) {
                    atomicOr(&c->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

// Queue tile (ty, tx) for sweep s unless it is queued already (one entry per
// tile per sweep: the stamp only grows).
__device__ __forceinline__ void push_tile(const PropParams &p, int ty, int tx, uint32_t s) {
    if (ty < 0 || tx < 0 || ty >= p.nty || tx >= p.ntx) return;
    const int t = ty * p.ntx + tx;
    if (atomicMax(p.queued + t, s + 1) < s + 1) {
        const uint32_t slot = s % 3;
        const uint32_t i = atomicAdd(&p.ctl->list_len[slot], 1u);
        p.lists[(size_t)slot * p.ntx * p.nty + i] = (uint32_t)t;
    }
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

// Persistent temporally blocked propagation. Block = NW warps; a row group is
// RXW consecutive lanes holding RXW consecutive words of R consecutive rows
// (one word per lane per row, in registers). Region = (NW * 32 / RXW * R) rows
// x RXW words; interior = rows [k, RY - k) x words [1, RXW - 1).
template <int RXW, int R, int NW, int MINB, typename DT>
__global__ void __launch_bounds__(NW * 32, MINB) k_propagate(PropParams p) {
    static_assert(RXW == 4 || RXW == 8 || RXW == 16 || RXW == 32, "row group width");
    static_assert(R >= 2, "rows per lane");
    constexpr int GPW = 32 / RXW;
    constexpr int G = NW * GPW;

    __shared__ uint32_t xtop[2][G][RXW];
    __shared__ uint32_t xbot[2][G][RXW];
    __shared__ int s_tile;
    __shared__ unsigned s_mask[2], s_done, s_maxl;   // s_mask by visit parity

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = lane % RXW;
    const int g = warp * GPW + lane / RXW;
    const int r0 = g * R;
    const int k = p.k, TY = p.TY, TXW = p.TXW;
    const int ntiles = p.ntx * p.nty;
    const GridDev &gd = p.g;
    DT *dist = reinterpret_cast<DT *>(gd.dist);
    const bool ownW = (w >= 1) && (w <= TXW);
    Ctl *ctl = p.ctl;
    unsigned thr_maxl = 0u;              // largest layer this thread's words reached
    unsigned long long blk_visits = 0;   // thread 0: tile visits of this block
    unsigned vq = 0u;                    // visit parity (block-uniform)

    // the seeding step rejected the targets (nothing in this kernel sets these
    // bits, so every block takes the same branch)
    if (ld_acquire(&ctl->err) & (ERR_INVAL | ERR_OBSTACLE)) return;

    const size_t ntl = (size_t)ntiles;
    for (uint32_t s = 0;; ++s) {
        const uint32_t l0 = s * (uint32_t)k;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            // slot (s + 2) % 3 last served sweep s - 1 and next serves s + 2
            ctl->work[(s + 2) % 3] = 0u;
            ctl->list_len[(s + 2) % 3] = 0u;
        }
        int jmax = k;
        if (p.max_layers && l0 + (uint32_t)k > p.max_layers) jmax = (int)(p.max_layers - l0);
        uint32_t *nbS = (s & 1) ? gd.nb1 : gd.nb0;
        const uint32_t *list = p.lists + (size_t)(s % 3) * ntl;
        unsigned *work = &ctl->work[s % 3];
        const uint32_t len = ld_acquire(&ctl->list_len[s % 3]);

        if (threadIdx.x == 0) {
            const uint32_t i = atomicAdd(work, 1u);
            s_tile = (i < len) ? (int)ld_relaxed(list + i) : -1;
        }
        __syncthreads();
        int t = s_tile;
        while (t >= 0) {
            // claim the next tile now; the atomic's latency hides behind this visit
            uint32_t next_i = 0;
            vq ^= 1u;
            if (threadIdx.x == 0) {
                next_i = atomicAdd(work, 1u);
                s_mask[vq] = 0u;   // last read two visits ago, before the previous visit's first barrier
            }

            // ---- load the region (tile + halo) ----
            const int ty = t / p.ntx, tx = t - ty * p.ntx;
            const int y0 = ty * TY - k;
            const int gw = tx * TXW - 1 + w;
            const bool inX = (gw >= 0) && (gw < gd.P);
            uint32_t V[R], F[R], NB[R], OWN[R];   // OWN: all-ones on this tile's interior words
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int rr = r0 + i, y = y0 + rr;
                const bool in = inX && y >= 0 && y < gd.H;
                const bool own = ownW && rr >= k && rr < k + TY;
                const size_t off = (size_t)y * gd.P + gw;
                OWN[i] = own ? 0xffffffffu : 0u;
                F[i] = in ? __ldg(gd.free_bits + off) : 0u;
                V[i] = in ? ld_relaxed(gd.vis + off) : 0u;
                NB[i] = 0u;
            }
            __threadfence();   // visit bits before the matching this-sweep bits
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (!OWN[i] && V[i]) V[i] &= ~ld_relaxed(nbS + (size_t)(y0 + r0 + i) * gd.P + gw);

            // ---- up to k layers in registers ----
            // P[b][i]: bit b of (layer - l0 - 1) for cells first reached in
            // this visit, so each cell's distance is written once, at the end.
            uint32_t P[5][R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
#pragma unroll
                for (int b = 0; b < 5; ++b) P[b][i] = 0u;
            }
            uint32_t changed = 1u;
            unsigned lastj = 0u;
            for (int j = 1; j <= jmax; ++j) {
                const uint32_t hF = hdil<RXW>(V[0]);
                const uint32_t hL = hdil<RXW>(V[R - 1]);
                xtop[j & 1][g][w] = hF;
                xbot[j & 1][g][w] = hL;
                if (!__syncthreads_or(changed != 0u)) break;   // region is stable
                const uint32_t hUp = (g > 0) ? xbot[j & 1][g - 1][w] : 0u;
                const uint32_t hDn = (g < G - 1) ? xtop[j & 1][g + 1][w] : 0u;
                uint32_t h[R];
                h[0] = hF;
                h[R - 1] = hL;
#pragma unroll
                for (int i = 1; i < R - 1; ++i) h[i] = hdil<RXW>(V[i]);
                uint32_t M[5];   // all-ones where bit b of j - 1 is set (block-uniform)
#pragma unroll
                for (int b = 0; b < 5; ++b) M[b] = (((j - 1) >> b) & 1) ? 0xffffffffu : 0u;
                changed = 0u;
                uint32_t own_new = 0u;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const uint32_t up = (i > 0) ? h[i - 1] : hUp;
                    const uint32_t dn = (i < R - 1) ? h[i + 1] : hDn;
                    const uint32_t nv = (up | h[i] | dn) & F[i] & ~V[i];
                    V[i] |= nv;
                    changed |= nv;
                    const uint32_t onv = nv & OWN[i];
                    NB[i] |= onv;
                    own_new |= onv;
#pragma unroll
                    for (int b = 0; b < 5; ++b) P[b][i] |= onv & M[b];
                }
                if (own_new) lastj = (unsigned)j;
            }

            // the claimed index has arrived by now; fetch its tile id early
            int next_t = -1;
            if (threadIdx.x == 0 && next_i < len) next_t = (int)ld_relaxed(list + next_i);

            // ---- frontier zones: cells reached at layer l0 + k ----
            uint32_t fmask = 0u;
            if (jmax == k) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    uint32_t last = NB[i];
#pragma unroll
                    for (int b = 0; b < 5; ++b)
                        last &= (((k - 1) >> b) & 1) ? P[b][i] : ~P[b][i];
                    fmask |= border_bits(r0 + i - k, w - 1, last, k, TY, TXW);
                }
            }
            if (fmask) atomicOr(&s_mask[vq], fmask);
            if (lastj) thr_maxl = max(thr_maxl, l0 + lastj);

            // ---- distances of the cells first reached in this visit ----
            // The warp writes one changed word at a time: 32 lanes, 32
            // consecutive cells, one coalesced store.
#pragma unroll
            for (int i = 0; i < R; ++i) {
                unsigned act = __ballot_sync(0xffffffffu, NB[i] != 0u);
                while (act) {
                    const int src = __ffs(act) - 1;
                    act &= act - 1u;
                    const uint32_t nb = __shfl_sync(0xffffffffu, NB[i], src);
                    uint32_t off = 0u;
#pragma unroll
                    for (int b = 0; b < 5; ++b)
                        off |= ((__shfl_sync(0xffffffffu, P[b][i], src) >> lane) & 1u) << b;
                    const int sw = src % RXW;                         // source word column
                    const int sg = warp * GPW + src / RXW;            // source row group
                    const int y = y0 + sg * R + i;
                    const int gws = tx * TXW - 1 + sw;
                    if ((nb >> lane) & 1u) {
                        const uint32_t layer = l0 + 1u + off;
                        if (sizeof(DT) == 2 && layer > 0xfffeu) atomicOr(&ctl->err, ERR_OVERFLOW);
                        else dist[(size_t)y * gd.W + (size_t)gws * 32 + lane] = (DT)layer;
                    }
                }
            }

            // ---- publish: this-sweep bits, then visit bits, then the queue ----
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (NB[i]) st_relaxed(nbS + (size_t)(y0 + r0 + i) * gd.P + gw, NB[i]);
            __threadfence();
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (NB[i]) st_relaxed(gd.vis + (size_t)(y0 + r0 + i) * gd.P + gw, V[i]);
            if (threadIdx.x == 0) {
                ++blk_visits;
                s_tile = next_t;
            }
            __syncthreads();
            if (threadIdx.x < 9) {
                // lanes 0..8 each queue one of the tiles the frontier reaches
                const uint32_t zone = 1u << threadIdx.x;
                if (s_mask[vq] & zone) push_reached(p, ty, tx, zone, s + 1);
            }
            t = s_tile;
        }

        if (!grid_barrier(ctl, gridDim.x, p.spin_limit)) return;
        if (threadIdx.x == 0) {
            // decided from values no block changes before the next barrier, so
            // every block reaches the same decision
            unsigned done = (ld_acquire(&ctl->list_len[(s + 1) % 3]) == 0u) ||
                            (p.max_layers && l0 + (uint32_t)k >= p.max_layers);
            if (!done && s + 1 >= p.sweep_cap) {
                atomicOr(&ctl->err, ERR_SWEEPS);
                done = 1;
            }
            if (done && blockIdx.x == 0) ctl->sweeps = s + 1;
            if (done && blk_visits) atomicAdd(&ctl->visits, blk_visits);
            s_done = done;
            s_maxl = 0u;
        }
        __syncthreads();
        if (s_done) {
            if (thr_maxl) atomicMax(&s_maxl, thr_maxl);
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
    atomicOr(g.vis + wo, bit);
    if (p.lists) {
        const int ty = y / p.TY, tx = (x >> 5) / p.TXW;
        const int ri = y - ty * p.TY, wi = (x >> 5) - tx * p.TXW;
        push_reached(p, ty, tx, border_bits(ri, wi, bit, p.k, p.TY, p.TXW), 0u);
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

template <int RXW, int R, int NW, int MINB>
void *variant_ptr(bool u16) {
    return u16 ? (void *)k_propagate<RXW, R, NW, MINB, uint16_t>
               : (void *)k_propagate<RXW, R, NW, MINB, uint32_t>;
}

// Compiled tile shapes: {region words, rows per lane, warps per block, blocks
// per SM the register budget aims at}. Region rows = warps * (32 / words) *
// rows per lane; interior = region minus k rows top and bottom and one word
// left and right.
constexpr VariantDesc kVariants[] = {
    {8, 4, 8, 3},    // 128 rows x 256 cells
    {8, 8, 8, 2},    // 256 rows x 256 cells
    {16, 4, 8, 3},   //  64 rows x 512 cells
    {4, 8, 8, 2},    // 512 rows x 128 cells
    {8, 4, 4, 5},    //  64 rows x 256 cells
    {16, 8, 8, 2},   // 128 rows x 512 cells
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
        default: return nullptr;
    }
}

}  // namespace

int num_variants() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }

VariantDesc variant_desc(int v) { return kVariants[v]; }

cudaError_t propagate_blocks_per_sm(int v, int dist_bits, int *out) {
    void *fn = variant_fn(v, dist_bits);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, kVariants[v].nwarps * 32, 0);
}

cudaError_t launch_propagate(int v, int dist_bits, const PropParams &p, int blocks,
                             cudaStream_t st) {
    void *fn = variant_fn(v, dist_bits);
    if (!fn) return cudaErrorInvalidValue;
    PropParams pp = p;
    void *args[] = {&pp};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kVariants[v].nwarps * 32), args, 0,
                                       st);
}

cudaError_t launch_seed(const uint32_t *targets, int n, const PropParams &p, int dist_bits,
                        cudaStream_t st) {
    const int tb = 256, nb = (n + tb - 1) / tb;
    count_launch();
    if (dist_bits == 16) k_seed<uint16_t><<<nb, tb, 0, st>>>(targets, n, p);
    else k_seed<uint32_t><<<nb, tb, 0, st>>>(targets, n, p);
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
