// Path reconstruction (Methods, "Path Reconstruction"): from a start, step to
// the neighbour with the largest activity -- on the distance plane, a
// neighbour with distance d - 1 -- until a target (d = 0). Ties go to the
// lowest linear index, i.e. the first of (dy,dx) = (-1,-1), (-1,0), (-1,1),
// (0,-1), (0,1), (1,-1), (1,0), (1,1).
//
// One warp per start. The walk is a chain of dependent steps, so its cost is
// load latency, not bandwidth: the warp loads a window of the distance plane
// around the current cell, then takes every step it can inside the window from
// shared memory (eight lanes test the eight neighbours, a ballot picks the
// first), and only reloads when the walk reaches the window's edge. uint32
// planes use 64 x 64 windows filled with asynchronous 4-byte copies (all 128
// per lane in flight at once, no registers held): a long walk crosses about
// half as many windows as with 32 x 32 ones, each about one memory round trip.
// Fewer such walks fit on the GPU at once, so the walks are taken longest
// first (k_order) and the longest ones start at once. uint16 planes use
// 32 x 32 windows of coalesced row loads.
#include <mutex>

#include <cuda_runtime.h>

#include "mpn_internal.cuh"

namespace mpn {

namespace {

constexpr int kWin = 32;          // window side (cells) of the Euclidean walk
constexpr int kWinPitch = 33;     // padded row pitch (bank spread)
constexpr int kTraceWarps = 4;    // warps per block

// walk windows: side, and warps per block (static shared memory <= 48 KB)
template <typename DT> struct TraceWin {
    static constexpr int side = 32, warps = 4;
};
template <> struct TraceWin<uint32_t> {
    static constexpr int side = 64, warps = 2;
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Walk order, longest paths first: one block sorts the starts into 33
// buckets by the bit length of their path length (a shared-memory count, a
// prefix, a scatter), so the walks of the longest bucket come first. Within a
// bucket the order is whatever the atomics give; it only affects speed.
__global__ void __launch_bounds__(1024) k_order(const uint64_t *__restrict__ offsets, int n,
                                                uint32_t *__restrict__ order) {
    __shared__ unsigned cnt[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0u;
    __syncthreads();
    auto bucket = [&](int i) {   // 0: length >= 2^31 ... 32: length 0
        const uint64_t len = offsets[i + 1] - offsets[i];
        const uint32_t l32 = len > 0xffffffffull ? 0xffffffffu : (uint32_t)len;
        return __clz(l32);
    };
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[bucket(i)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0u;
        for (int k = 0; k < 33; ++k) {
            const unsigned c = cnt[k];
            cnt[k] = a;
            a += c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[atomicAdd(&cnt[bucket(i)], 1u)] = (uint32_t)i;
}

template <typename DT>
__global__ void k_lengths(GridDev g, const uint32_t *__restrict__ starts, int n,
                          uint64_t *__restrict__ offsets, int8_t *__restrict__ status,
                          uint32_t *err, uint32_t *walk_max) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) offsets[0] = 0ull;
    if (i >= n) return;
    const uint32_t s = starts[i];
    uint64_t len = 0;
    int8_t stt = MPN_PATH_OK;
    if ((uint64_t)s >= (uint64_t)g.H * (uint64_t)g.W) {
        atomicOr(err, ERR_INVAL);
        stt = MPN_PATH_UNREACHABLE;
    } else {
        const int y = (int)(s / (uint32_t)g.W), x = (int)(s % (uint32_t)g.W);
        const DT d = reinterpret_cast<const DT *>(g.dist)[s];
        if (!((g.free_bits[(size_t)y * g.P + (x >> 5)] >> (x & 31)) & 1u)) stt = MPN_PATH_ON_OBSTACLE;
        else if (d == (DT)~(DT)0) stt = MPN_PATH_UNREACHABLE;
        else len = (uint64_t)d + 1u;
    }
    offsets[i + 1] = len;
    status[i] = stt;
    // the longest path, one atomic per warp
    const uint32_t m = __reduce_max_sync(__activemask(), len > 0xffffffffull ? 0xffffffffu : (uint32_t)len);
    if ((threadIdx.x & 31) == __ffs(__activemask()) - 1 && m) atomicMax(walk_max, m);
}

// In-place inclusive scan of a[1..n] by one block: chunks of blockDim * 8
// elements, each thread summing 8 consecutive values, a warp-shuffle scan over
// thread sums, and a running carry across chunks.
__device__ __forceinline__ void block_scan_inplace(uint64_t *a, int n) {
    constexpr int ITEMS = 8;
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    if (tid == 0) carry_s = 0ull;
    __syncthreads();
    uint64_t *x = a + 1;
    for (int base = 0; base < n; base += blockDim.x * ITEMS) {
        uint64_t v[ITEMS];
        uint64_t sum = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = base + tid * ITEMS + j;
            v[j] = (idx < n) ? x[idx] : 0ull;
            sum += v[j];
        }
        uint64_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint64_t wt = (lane < nw) ? warp_tot[lane] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t t = __shfl_up_sync(0xffffffffu, wt, o);
                if (lane >= o) wt += t;
            }
            if (lane < nw) warp_tot[lane] = wt;
        }
        __syncthreads();
        uint64_t run = carry_s + (wid > 0 ? warp_tot[wid - 1] : 0ull) + (inc - sum);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = base + tid * ITEMS + j;
            run += v[j];
            if (idx < n) x[idx] = run;
        }
        __syncthreads();
        if (tid == 0) carry_s += warp_tot[nw - 1];
        __syncthreads();
    }
}

__global__ void k_scan(uint64_t *a, int n) { block_scan_inplace(a, n); }

// One walk by the calling warp (all 32 lanes), from cell c (free, reached)
// down to distance dstop (0: a target). wb: the warp's window buffer, kW x
// (kW + 1) elements of DT. CELLS: the walk's cells go to cells[o0], cells[o0 +
// 1], ...; *end gets the linear index of the cell the walk ends at. False if
// the plane is not a distance plane (no neighbour one step closer; ERR_TRACE
// recorded).
template <typename DT, int kW, bool CELLS>
__device__ __forceinline__ bool walk_path(const GridDev &g, uint32_t c, uint64_t o0, DT *wb,
                                          uint32_t *__restrict__ cells, uint32_t *err, uint32_t *end,
                                          uint32_t dstop = 0u) {
    constexpr int kP = kW + 1;
    const int lane = threadIdx.x & 31;
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    const DT INF = (DT)~(DT)0;
    // neighbour of lane q (q < 8) in the tie-break order
    const int my_dy = (lane < 3) ? -1 : (lane < 5 ? 0 : 1);
    const int my_dx = (lane == 0 || lane == 3 || lane == 5) ? -1 : ((lane == 1 || lane == 6) ? 0 : 1);
    // two-step lookahead: this lane's first step q1 = lane / 4 and second
    // steps q2 = lane % 4, lane % 4 + 4 (offsets from the same packed tables)
    const int q1l = lane >> 2, q2a = lane & 3, q2b = q2a + 4;
    const int dy1 = (int)((0xa940u >> (2 * q1l)) & 3u) - 1, dx1 = (int)((0x9224u >> (2 * q1l)) & 3u) - 1;
    const int dy2a = (int)((0xa940u >> (2 * q2a)) & 3u) - 1, dx2a = (int)((0x9224u >> (2 * q2a)) & 3u) - 1;
    const int dy2b = (int)((0xa940u >> (2 * q2b)) & 3u) - 1, dx2b = (int)((0x9224u >> (2 * q2b)) & 3u) - 1;
    // the same as offsets in the window (row pitch kP), from the current cell
    const int off1 = dy1 * kP + dx1;
    const int off2a = off1 + dy2a * kP + dx2a, off2b = off1 + dy2b * kP + dx2b;
    const int my_off = my_dy * kP + my_dx;

    uint64_t o = o0;
    int cy = (int)(c / (uint32_t)g.W), cx = (int)(c % (uint32_t)g.W);
    uint32_t d = (uint32_t)dist[c];
    if (CELLS && lane == 0) cells[o] = c;
    int ddy = 0, ddx = 0;   // how far the walk moved in the last window
    while (d > dstop) {
        // the next window reaches further in the direction the walk has been
        // heading: along an axis on which it moved at least kW / 4 cells in
        // the last window, the current cell sits a quarter window in from the
        // trailing edge; otherwise it is centred
        const int oy = ddy >= kW / 4 ? kW / 4 : (ddy <= -kW / 4 ? kW - 1 - kW / 4 : kW / 2);
        const int ox = ddx >= kW / 4 ? kW / 4 : (ddx <= -kW / 4 ? kW - 1 - kW / 4 : kW / 2);
        const int wy0 = cy - oy, wx0 = cx - ox;
        if (sizeof(DT) == 4) {
#pragma unroll 4
            for (int r = 0; r < kW; ++r) {
                const int y = wy0 + r;
#pragma unroll
                for (int u = 0; u < kW / 32; ++u) {
                    const int x = wx0 + 32 * u + lane;
                    DT *sp = wb + r * kP + 32 * u + lane;
                    if (y >= 0 && y < g.H && x >= 0 && x < g.W) cp_async4(sp, dist + (size_t)y * g.W + x);
                    else *sp = INF;
                }
            }
            cp_async_wait_all();
        } else {
            const int x = wx0 + lane;
#pragma unroll 8
            for (int r = 0; r < kW; ++r) {
                const int y = wy0 + r;
                DT v = INF;
                if (y >= 0 && y < g.H && x >= 0 && x < g.W) v = dist[(size_t)y * g.W + x];
                wb[r * kP + lane] = v;
            }
        }
        __syncwarp();
        int ly = oy, lx = ox;
        while (d > dstop && ly >= 1 && ly <= kW - 2 && lx >= 1 && lx <= kW - 2) {
            if (d >= dstop + 2u && ly >= 2 && ly <= kW - 3 && lx >= 2 && lx <= kW - 3) {
                // two steps at once: lane L tests first step q1 = L / 4 (a
                // d - 1 neighbour) and second steps q2 = L % 4 and L % 4 + 4
                // from there (d - 2 neighbours); the first valid q1 in
                // tie-break order, then its first valid q2, are the two steps
                // the single-step rule takes
                const DT *cur = wb + ly * kP + lx;
                const bool a = (uint32_t)cur[off1] == d - 1u;
                const bool b0 = (uint32_t)cur[off2a] == d - 2u;
                const bool b1 = (uint32_t)cur[off2b] == d - 2u;
                const unsigned m1 = __ballot_sync(0xffffffffu, a);
                const unsigned ma = __ballot_sync(0xffffffffu, a && b0);
                const unsigned mb = __ballot_sync(0xffffffffu, a && b1);
                if (!m1) {                      // not a distance plane: give up on this path
                    if (lane == 0) atomicOr(err, ERR_TRACE);
                    return false;
                }
                const int g1 = (__ffs(m1) - 1) & ~3;   // 4 * q1
                const unsigned m2 = ((ma >> g1) & 0xfu) | (((mb >> g1) & 0xfu) << 4);
                if (!m2) {
                    if (lane == 0) atomicOr(err, ERR_TRACE);
                    return false;
                }
                const int q1 = g1 >> 2, q2 = __ffs(m2) - 1;
                const int ly1 = ly + (int)((0xa940u >> (2 * q1)) & 3u) - 1;
                const int lx1 = lx + (int)((0x9224u >> (2 * q1)) & 3u) - 1;
                ly = ly1 + (int)((0xa940u >> (2 * q2)) & 3u) - 1;
                lx = lx1 + (int)((0x9224u >> (2 * q2)) & 3u) - 1;
                d -= 2u;
                if (CELLS && lane == 0) {
                    cells[o + 1] = (uint32_t)((wy0 + ly1) * g.W + (wx0 + lx1));
                    cells[o + 2] = (uint32_t)((wy0 + ly) * g.W + (wx0 + lx));
                }
                o += 2;
                continue;
            }
            bool hit = false;
            if (lane < 8) hit = (uint32_t)wb[ly * kP + lx + my_off] == d - 1u;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (!m) {                      // not a distance plane: give up on this path
                if (lane == 0) atomicOr(err, ERR_TRACE);
                return false;
            }
            // neighbour q's offsets from two packed tables (2 bits per q:
            // offset + 1), the same order as my_dy / my_dx
            const int q = __ffs(m) - 1;
            ly += (int)((0xa940u >> (2 * q)) & 3u) - 1;
            lx += (int)((0x9224u >> (2 * q)) & 3u) - 1;
            --d;
            ++o;
            if (CELLS && lane == 0) cells[o] = (uint32_t)((wy0 + ly) * g.W + (wx0 + lx));
        }
        __syncwarp();
        ddy = ly - oy;
        ddx = lx - ox;
        cy = wy0 + ly;
        cx = wx0 + lx;
    }
    *end = (uint32_t)cy * (uint32_t)g.W + (uint32_t)cx;
    return true;
}

// CELLS: write the whole path at offsets[i]; otherwise write only the cell
// the walk ends at (the target reached) to ends[i] and the start's distance
// to ends_d[i] (0xFFFFFFFF for both when the start has no path).
template <typename DT, bool CELLS>
__global__ void __launch_bounds__(TraceWin<DT>::warps * 32)
    k_trace(GridDev g, const uint32_t *__restrict__ starts, int n,
            const uint64_t *__restrict__ offsets, const int8_t *__restrict__ status,
            uint32_t *__restrict__ cells, uint32_t *__restrict__ ends, uint32_t *__restrict__ ends_d,
            uint32_t *err, const uint32_t *__restrict__ order, uint64_t skip_above = ~0ull) {
    constexpr int kW = TraceWin<DT>::side, kP = kW + 1, NWp = TraceWin<DT>::warps;
    __shared__ DT win[NWp][kW * kP];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int slot = blockIdx.x * NWp + wl;
    if (slot >= n) return;                      // whole warp leaves together
    const int i = order ? (int)order[slot] : slot;
    if (i < 0 || i >= n) return;
    if (status[i] != MPN_PATH_OK) {
        if (!CELLS && lane == 0) {
            ends[i] = 0xffffffffu;
            if (ends_d) ends_d[i] = 0xffffffffu;
        }
        return;
    }
    if (CELLS && offsets[i + 1] - offsets[i] > skip_above) return;   // walked in segments
    const uint32_t c = starts[i];
    const uint32_t d0 = (uint32_t)reinterpret_cast<const DT *>(g.dist)[c];
    uint32_t e = 0;
    if (!walk_path<DT, kW, CELLS>(g, c, CELLS ? offsets[i] : 0ull, win[wl], cells, err, &e)) return;
    if (!CELLS && lane == 0) {
        ends[i] = e;
        if (ends_d) ends_d[i] = d0;
    }
}

// ---- on-device invariant check of a distance plane ----

// Cells breaking what a multi-source, 8-connected, unit-cost distance map
// must satisfy: a reached cell at d > 0 without a free neighbour at d - 1;
// two reached neighbours more than 1 apart; a reached cell below the layer
// cap (M, 0 = none) next to an unreached free cell; an obstacle marked
// reached. Warp-aggregated count.
template <typename DT>
__global__ void k_check_plane(GridDev g, uint32_t M, unsigned long long *count) {
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    const DT INF = (DT)~(DT)0;
    const size_t n = (size_t)g.H * g.W;
    unsigned bad = 0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / (size_t)g.W), x = (int)(c % (size_t)g.W);
        const bool free = (g.free_bits[(size_t)y * g.P + (x >> 5)] >> (x & 31)) & 1u;
        const DT d = dist[c];
        if (!free) {
            bad += d != INF;
            continue;
        }
        if (d == INF) continue;   // its reached neighbours check the pair
        bool down = d == (DT)0, ok = true;
        for (int q = 0; q < 8; ++q) {
            const int yy = y + (int)((0xa940u >> (2 * q)) & 3u) - 1;
            const int xx = x + (int)((0x9224u >> (2 * q)) & 3u) - 1;
            if (yy < 0 || xx < 0 || yy >= g.H || xx >= g.W) continue;
            if (!((g.free_bits[(size_t)yy * g.P + (xx >> 5)] >> (xx & 31)) & 1u)) continue;
            const DT e = dist[(size_t)yy * g.W + xx];
            if (e == INF) {
                if (!M || (uint32_t)d < M) ok = false;
            } else {
                if ((uint32_t)e + 1u < (uint32_t)d || (uint32_t)d + 1u < (uint32_t)e) ok = false;
                if ((uint32_t)e + 1u == (uint32_t)d) down = true;
            }
        }
        bad += !(ok && down);
    }
    const unsigned tot = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(count, (unsigned long long)tot);
}

// ---- long walks in segments ----

// succ[c] = the next cell of the walk from c (the first neighbour in
// tie-break order with distance d - 1), c itself for targets, unreached cells
// and obstacles.
template <typename DT>
__global__ void k_succ(GridDev g, uint32_t *__restrict__ succ) {
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    const DT INF = (DT)~(DT)0;
    const size_t n = (size_t)g.H * g.W;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const DT d = dist[c];
        uint32_t nx = (uint32_t)c;
        if (d != INF && d != (DT)0) {
            const int y = (int)(c / (size_t)g.W), x = (int)(c % (size_t)g.W);
            for (int q = 0; q < 8; ++q) {
                const int yy = y + (int)((0xa940u >> (2 * q)) & 3u) - 1;
                const int xx = x + (int)((0x9224u >> (2 * q)) & 3u) - 1;
                if (yy < 0 || xx < 0 || yy >= g.H || xx >= g.W) continue;
                const size_t o = (size_t)yy * g.W + xx;
                if (dist[o] == (DT)(d - 1)) {
                    nx = (uint32_t)o;
                    break;
                }
            }
        }
        succ[c] = nx;
    }
}

// out = in o in (one squaring of the jump table)
__global__ void k_square(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t n) {
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        out[c] = in[in[c]];
}

// Thread per start: a walk longer than kLongWalk cells becomes segments of
// kSegLen steps (the last one shorter); their first cells are kSegLen apart
// along the walk, read from the jump table.
template <typename DT>
__global__ void k_segments(GridDev g, const uint32_t *__restrict__ starts, int n,
                           const uint64_t *__restrict__ offsets, const int8_t *__restrict__ status,
                           const uint32_t *__restrict__ jump, WalkSeg *__restrict__ segs, uint32_t cap,
                           uint32_t *nseg, uint32_t *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || status[i] != MPN_PATH_OK) return;
    const uint64_t o = offsets[i];
    if (offsets[i + 1] - o <= kLongWalk) return;
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    uint32_t c = starts[i];
    uint32_t d = (uint32_t)dist[c];
    for (uint64_t k = 0;; ++k) {
        const uint32_t dstop = d > kSegLen ? d - kSegLen : 0u;
        const uint32_t idx = atomicAdd(nseg, 1u);
        if (idx >= cap) {   // (the caller sizes the room; defensive)
            atomicOr(err, ERR_TRACE);
            return;
        }
        segs[idx] = WalkSeg{c, dstop, o + k * kSegLen};
        if (dstop == 0u) return;
        c = jump[c];
        if ((uint32_t)dist[c] != dstop) {   // not a distance plane
            atomicOr(err, ERR_TRACE);
            return;
        }
        d = dstop;
    }
}

// Warp per segment: the walk from its first cell down to its stop distance.
template <typename DT>
__global__ void __launch_bounds__(TraceWin<DT>::warps * 32)
    k_trace_segs(GridDev g, const WalkSeg *__restrict__ segs, const uint32_t *__restrict__ nseg,
                 uint32_t *__restrict__ cells, uint32_t *err) {
    constexpr int kW = TraceWin<DT>::side, kP = kW + 1, NWp = TraceWin<DT>::warps;
    __shared__ DT win[NWp][kW * kP];
    const int wl = threadIdx.x >> 5;
    const uint32_t j = blockIdx.x * NWp + wl;
    if (j >= *nseg) return;
    const WalkSeg sg = segs[j];
    uint32_t e = 0;
    walk_path<DT, kW, true>(g, sg.cell, sg.out, win[wl], cells, err, &e, sg.dstop);
}

// ---- batched trace over the grids of a batch ----

// One block per job: the status and length of every start (as k_lengths),
// the offsets scanned in place, the job's total, and the flat walk lengths.
__global__ void __launch_bounds__(256) k_lengths_batch(const WalkJob *__restrict__ jobs,
                                                       uint32_t *__restrict__ walk_len,
                                                       uint64_t *__restrict__ totals, uint32_t *err) {
    __shared__ uint32_t s_max;
    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    const WalkJob jb = jobs[blockIdx.x];
    const GridDev &g = jb.g;
    const uint64_t N = (uint64_t)g.H * (uint64_t)g.W;
    if (threadIdx.x == 0) jb.offsets[0] = 0ull;
    for (uint32_t i = threadIdx.x; i < jb.ns; i += blockDim.x) {
        const uint32_t s = jb.starts[i];
        uint64_t len = 0;
        int8_t stt = MPN_PATH_OK;
        if ((uint64_t)s >= N) {
            atomicOr(err, ERR_INVAL);
            stt = MPN_PATH_UNREACHABLE;
        } else {
            const int y = (int)(s / (uint32_t)g.W), x = (int)(s % (uint32_t)g.W);
            const uint32_t d = jb.dist_bits == 16 ? (uint32_t)reinterpret_cast<const uint16_t *>(g.dist)[s]
                                                  : reinterpret_cast<const uint32_t *>(g.dist)[s];
            const uint32_t inf = jb.dist_bits == 16 ? 0xffffu : 0xffffffffu;
            if (!((g.free_bits[(size_t)y * g.P + (x >> 5)] >> (x & 31)) & 1u)) stt = MPN_PATH_ON_OBSTACLE;
            else if (d == inf) stt = MPN_PATH_UNREACHABLE;
            else len = (uint64_t)d + 1u;
        }
        jb.offsets[i + 1] = len;
        jb.status[i] = stt;
        const uint32_t l32 = len > 0xffffffffull ? 0xffffffffu : (uint32_t)len;
        walk_len[jb.walk_base + i] = l32;
        if (l32) atomicMax(&s_max, l32);
    }
    __syncthreads();
    block_scan_inplace(jb.offsets, (int)jb.ns);
    if (threadIdx.x == 0) {
        totals[blockIdx.x] = jb.offsets[jb.ns];
        totals[gridDim.x + blockIdx.x] = s_max;
    }
}

// Walk order over flat lengths, longest first (as k_order).
__global__ void __launch_bounds__(1024) k_order_len(const uint32_t *__restrict__ len, uint32_t n,
                                                    uint32_t *__restrict__ order) {
    __shared__ unsigned cnt[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[__clz(len[i])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0u;
        for (int k = 0; k < 33; ++k) {
            const unsigned c = cnt[k];
            cnt[k] = a;
            a += c;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) order[atomicAdd(&cnt[__clz(len[i])], 1u)] = i;
}

// Warp per walk over every job: the walk's job is the last one whose first
// walk index is not above it (jobs are in walk order). A batch's walks are
// many (their total, not the longest one, sets the time), so they use 32 x 32
// windows for both dtypes: four times as many walks fit on the GPU at once as
// with the single-grid trace's 64 x 64 uint32 windows.
constexpr int kBatchTraceWarps = 8;
constexpr int kBatchWin = 32;
__global__ void __launch_bounds__(kBatchTraceWarps * 32)
    k_trace_batch(const WalkJob *__restrict__ jobs, int njobs, const uint32_t *__restrict__ order,
                  uint32_t nwalks, uint32_t *err) {
    __shared__ __align__(16) uint32_t win[kBatchTraceWarps][kBatchWin * (kBatchWin + 1)];
    const int wl = threadIdx.x >> 5;
    const uint32_t slot = blockIdx.x * kBatchTraceWarps + wl;
    if (slot >= nwalks) return;                 // whole warp leaves together
    const uint32_t w = order[slot];
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].walk_base <= w) lo = mid;
        else hi = mid - 1;
    }
    const WalkJob &jb = jobs[lo];
    const uint32_t i = w - jb.walk_base;
    if (i >= jb.ns || !jb.cells || jb.status[i] != MPN_PATH_OK) return;
    if (jb.split && jb.offsets[i + 1] - jb.offsets[i] > kLongWalk) return;   // walked in segments
    uint32_t e = 0;
    if (jb.dist_bits == 16)
        walk_path<uint16_t, kBatchWin, true>(jb.g, jb.starts[i], jb.offsets[i],
                                             reinterpret_cast<uint16_t *>(win[wl]), jb.cells, err, &e);
    else
        walk_path<uint32_t, kBatchWin, true>(jb.g, jb.starts[i], jb.offsets[i], win[wl], jb.cells, err, &e);
}

// Thread per start of batch job j: its walk, if longer than kLongWalk cells,
// becomes segments (as k_segments) tagged with the job.
template <typename DT>
__global__ void k_segments_batch(const WalkJob *__restrict__ jobs, int j, const uint32_t *__restrict__ jump,
                                 BatchSeg *__restrict__ segs, uint32_t cap, uint32_t *nseg, uint32_t *err) {
    const WalkJob &jb = jobs[j];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= jb.ns || jb.status[i] != MPN_PATH_OK) return;
    const uint64_t o = jb.offsets[i];
    if (jb.offsets[i + 1] - o <= kLongWalk) return;
    const DT *dist = reinterpret_cast<const DT *>(jb.g.dist);
    uint32_t c = jb.starts[i];
    uint32_t d = (uint32_t)dist[c];
    for (uint64_t k = 0;; ++k) {
        const uint32_t dstop = d > kSegLen ? d - kSegLen : 0u;
        const uint32_t idx = atomicAdd(nseg, 1u);
        if (idx >= cap) {
            atomicOr(err, ERR_TRACE);
            return;
        }
        segs[idx] = BatchSeg{c, dstop, (uint32_t)j, 0u, o + k * kSegLen};
        if (dstop == 0u) return;
        c = jump[c];
        if ((uint32_t)dist[c] != dstop) {
            atomicOr(err, ERR_TRACE);
            return;
        }
        d = dstop;
    }
}

// Warp per segment of any job (32 x 32 windows, as k_trace_batch).
__global__ void __launch_bounds__(kBatchTraceWarps * 32)
    k_trace_segs_batch(const WalkJob *__restrict__ jobs, const BatchSeg *__restrict__ segs,
                       const uint32_t *__restrict__ nseg, uint32_t *err) {
    __shared__ __align__(16) uint32_t win[kBatchTraceWarps][kBatchWin * (kBatchWin + 1)];
    const int wl = threadIdx.x >> 5;
    const uint32_t q = blockIdx.x * kBatchTraceWarps + wl;
    if (q >= *nseg) return;
    const BatchSeg sg = segs[q];
    const WalkJob &jb = jobs[sg.job];
    uint32_t e = 0;
    if (jb.dist_bits == 16)
        walk_path<uint16_t, kBatchWin, true>(jb.g, sg.cell, sg.out, reinterpret_cast<uint16_t *>(win[wl]),
                                             jb.cells, err, &e, sg.dstop);
    else
        walk_path<uint32_t, kBatchWin, true>(jb.g, sg.cell, sg.out, win[wl], jb.cells, err, &e, sg.dstop);
}

// Euclidean path reconstruction (Eq. 1 and the straightening rule after it),
// one warp per start, in the same 32 x 32 shared-memory windows as k_trace.
// Each step tests all candidate moves at once: lanes 0-3 the 4-neighbours in
// Eq. 1's order (left, right, up, down) for distance d - 1; lanes 4-19 the
// corner rule (4-neighbour q with distance d that is 4-adjacent, through r,
// to a cell with d - 1); lanes 20-27 the 8-neighbours for d - 1 (both corners
// blocked). The first hit in that order is taken. Straightening runs on the
// fly with a one-point delay: a point is dropped when the last kept point and
// the next point are sqrt(2) apart. COUNT pass: only the kept length; WRITE
// pass: the cells at the offsets of the count pass.
template <typename DT, bool WRITE>
__global__ void __launch_bounds__(kTraceWarps * 32)
    k_euclid(GridDev g, const uint32_t *__restrict__ starts, int n, uint64_t *__restrict__ offsets,
             const int8_t *__restrict__ status, uint32_t *__restrict__ cells, uint32_t *err) {
    __shared__ DT win[kTraceWarps][kWin * kWinPitch];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int i = blockIdx.x * kTraceWarps + wl;
    if (i >= n) return;
    if (status[i] != MPN_PATH_OK) {
        if (!WRITE && lane == 0) offsets[i + 1] = 0ull;
        return;
    }
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    const DT INF = (DT)~(DT)0;
    DT *wb = win[wl];
    // per-lane candidate geometry: (qy, qx) first move, (ry, rx) second
    int qy = 0, qx = 0, ry = 0, rx = 0;
    {
        const int EY[4] = {0, 0, -1, 1}, EX[4] = {-1, 1, 0, 0};
        const int DY8[8] = {-1, -1, -1, 0, 0, 1, 1, 1}, DX8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
        if (lane < 4) { qy = EY[lane]; qx = EX[lane]; }
        else if (lane < 20) { qy = EY[(lane - 4) >> 2]; qx = EX[(lane - 4) >> 2];
                              ry = EY[(lane - 4) & 3]; rx = EX[(lane - 4) & 3]; }
        else if (lane < 28) { qy = DY8[lane - 20]; qx = DX8[lane - 20]; }
    }
    const uint32_t s0 = starts[i];
    uint64_t o = WRITE ? offsets[i] : 0ull;
    uint64_t kept = 0;
    int cy = (int)(s0 / (uint32_t)g.W), cx = (int)(s0 % (uint32_t)g.W);
    uint32_t d = (uint32_t)dist[s0];
    // straightening state: last kept point, pending point
    int ky = cy, kx = cx, py = -1, px = -1;
    bool has_pending = false;
    if (WRITE && lane == 0) cells[o] = s0;
    ++kept;
    while (d > 0) {
        const int wy0 = cy - kWin / 2, wx0 = cx - kWin / 2;
        const int x = wx0 + lane;
#pragma unroll 8
        for (int r = 0; r < kWin; ++r) {
            const int y = wy0 + r;
            DT v = INF;
            if (y >= 0 && y < g.H && x >= 0 && x < g.W) v = dist[(size_t)y * g.W + x];
            wb[r * kWinPitch + lane] = v;
        }
        __syncwarp();
        int ly = cy - wy0, lx = cx - wx0;
        while (d > 0 && ly >= 2 && ly <= kWin - 3 && lx >= 2 && lx <= kWin - 3) {
            bool hit = false;
            if (lane < 4 || (lane >= 20 && lane < 28)) {
                hit = (uint32_t)wb[(ly + qy) * kWinPitch + lx + qx] == d - 1u;
            } else if (lane < 20) {
                hit = (uint32_t)wb[(ly + qy) * kWinPitch + lx + qx] == d &&
                      (uint32_t)wb[(ly + qy + ry) * kWinPitch + lx + qx + rx] == d - 1u;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            unsigned pick = m & 0xfu;
            if (!pick) pick = m & 0xffff0u;
            if (!pick) pick = m & 0x0ff00000u;
            if (!pick) {
                if (lane == 0) atomicOr(err, ERR_TRACE);
                return;
            }
            const int q = __ffs(pick) - 1;
            const int sy = __shfl_sync(0xffffffffu, qy, q), sx = __shfl_sync(0xffffffffu, qx, q);
            ly += sy;
            lx += sx;
            if (q < 4 || q >= 20) --d;   // a corner move keeps the distance
            // straightening with a one-point delay
            const int ny = wy0 + ly, nx = wx0 + lx;
            if (has_pending) {
                const int ay = ky - ny, ax = kx - nx;
                if (ay * ay + ax * ax != 2) {      // keep the pending point
                    if (WRITE && lane == 0) cells[o + kept] = (uint32_t)(py * g.W + px);
                    ++kept;
                    ky = py;
                    kx = px;
                }
            }
            py = ny;
            px = nx;
            has_pending = true;
        }
        __syncwarp();
        cy = wy0 + ly;
        cx = wx0 + lx;
    }
    if (has_pending) {   // the last point (a target) is always kept
        if (WRITE && lane == 0) cells[o + kept] = (uint32_t)(py * g.W + px);
        ++kept;
    }
    if (!WRITE && lane == 0) offsets[i + 1] = kept;
}

template <typename DT>
__global__ void k_activity(GridDev g, uint32_t L, int32_t *out) {
    const DT *dist = reinterpret_cast<const DT *>(g.dist);
    const size_t n = (size_t)g.H * g.W;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const DT d = dist[i];
        out[i] = (d != (DT)~(DT)0 && (uint32_t)d <= L) ? (int32_t)(L + 1u - (uint32_t)d) : 0;
    }
}

int grid_for(size_t work_items, int per_block) {
    size_t b = (work_items + per_block - 1) / per_block;
    if (b > (size_t)152 * 32) b = (size_t)152 * 32;
    return (int)(b ? b : 1);
}

}  // namespace

cudaError_t launch_trace_lengths(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                                 uint64_t *offsets, int8_t *status, Ctl *ctl, cudaStream_t st) {
    const int tb = 256, nb = (n + 1 + tb - 1) / tb;
    count_launch();
    if (dist_bits == 16) k_lengths<uint16_t><<<nb, tb, 0, st>>>(g, starts, n, offsets, status, &ctl->err, &ctl->walk_max);
    else k_lengths<uint32_t><<<nb, tb, 0, st>>>(g, starts, n, offsets, status, &ctl->err, &ctl->walk_max);
    return cudaGetLastError();
}

cudaError_t launch_scan(uint64_t *offsets, int n, cudaStream_t st) {
    count_launch();
    k_scan<<<1, 1024, 0, st>>>(offsets, n);
    return cudaGetLastError();
}

// the largest shared-memory carveout for the 64 x 64 windows
static cudaError_t trace_attributes() {
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
        const void *fns[2] = {(const void *)k_trace<uint32_t, true>, (const void *)k_trace<uint32_t, false>};
        for (const void *f : fns)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    });
    return e;
}

cudaError_t launch_trace(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                         const uint64_t *offsets, const int8_t *status, uint32_t *cells,
                         uint32_t *order, cudaStream_t st, uint32_t *err) {
    if (n <= 0) return cudaSuccess;
    if (cudaError_t e = trace_attributes()) return e;
    if (dist_bits == 16) {
        constexpr int w = TraceWin<uint16_t>::warps;
        count_launch();
        k_trace<uint16_t, true><<<(n + w - 1) / w, w * 32, 0, st>>>(g, starts, n, offsets, status, cells,
                                                                    nullptr, nullptr, err, nullptr);
    } else {
        constexpr int w = TraceWin<uint32_t>::warps;
        const uint32_t *ord = nullptr;
        if (order) {
            count_launch();
            k_order<<<1, 1024, 0, st>>>(offsets, n, order);
            ord = order;
        }
        count_launch();
        k_trace<uint32_t, true><<<(n + w - 1) / w, w * 32, 0, st>>>(g, starts, n, offsets, status, cells,
                                                                    nullptr, nullptr, err, ord);
    }
    return cudaGetLastError();
}

cudaError_t launch_check_plane(const GridDev &g, int dist_bits, uint32_t max_layers,
                               unsigned long long *count, cudaStream_t st) {
    const size_t n = (size_t)g.H * g.W;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    count_launch();
    if (dist_bits == 16) k_check_plane<uint16_t><<<grid_for(n, 256), 256, 0, st>>>(g, max_layers, count);
    else k_check_plane<uint32_t><<<grid_for(n, 256), 256, 0, st>>>(g, max_layers, count);
    return cudaGetLastError();
}

cudaError_t launch_jump_table(const GridDev &g, int dist_bits, uint32_t *jump, uint32_t **table,
                              cudaStream_t st) {
    const size_t cells_n = (size_t)g.H * g.W;
    uint32_t *a = jump, *b = jump + cells_n;
    const int nb = grid_for(cells_n, 256);
    count_launch();
    if (dist_bits == 16) k_succ<uint16_t><<<nb, 256, 0, st>>>(g, a);
    else k_succ<uint32_t><<<nb, 256, 0, st>>>(g, a);
    for (uint32_t m = 1; m < kSegLen; m *= 2) {   // a = succ^m -> succ^(2m)
        count_launch();
        k_square<<<nb, 256, 0, st>>>(a, b, cells_n);
        uint32_t *t = a;
        a = b;
        b = t;
    }
    *table = a;
    return cudaGetLastError();
}

cudaError_t launch_batch_segments(const WalkJob *jobs, int j, uint32_t ns, int dist_bits,
                                  const uint32_t *table, BatchSeg *segs, uint32_t cap, uint32_t *nseg,
                                  uint32_t *err, cudaStream_t st) {
    if (ns == 0) return cudaSuccess;
    count_launch();
    if (dist_bits == 16)
        k_segments_batch<uint16_t><<<(ns + 255) / 256, 256, 0, st>>>(jobs, j, table, segs, cap, nseg, err);
    else
        k_segments_batch<uint32_t><<<(ns + 255) / 256, 256, 0, st>>>(jobs, j, table, segs, cap, nseg, err);
    return cudaGetLastError();
}

cudaError_t launch_batch_segwalks(const WalkJob *jobs, const BatchSeg *segs, const uint32_t *nseg,
                                  uint32_t cap, uint32_t *err, cudaStream_t st) {
    if (cap == 0) return cudaSuccess;
    count_launch();
    k_trace_segs_batch<<<(cap + kBatchTraceWarps - 1) / kBatchTraceWarps, kBatchTraceWarps * 32, 0, st>>>(
        jobs, segs, nseg, err);
    return cudaGetLastError();
}

cudaError_t launch_trace_split(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                               const uint64_t *offsets, const int8_t *status, uint32_t *cells,
                               uint32_t *order, uint32_t *jump, WalkSeg *segs, uint32_t seg_cap,
                               uint32_t *nseg, cudaStream_t st, uint32_t *err) {
    if (n <= 0) return cudaSuccess;
    if (cudaError_t e = trace_attributes()) return e;
    cudaError_t e = cudaMemsetAsync(nseg, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    uint32_t *a = nullptr;
    if ((e = launch_jump_table(g, dist_bits, jump, &a, st)) != cudaSuccess) return e;
    const int tb = 256;
    count_launch(3);
    if (dist_bits == 16)
        k_segments<uint16_t><<<(n + tb - 1) / tb, tb, 0, st>>>(g, starts, n, offsets, status, a, segs, seg_cap, nseg, err);
    else
        k_segments<uint32_t><<<(n + tb - 1) / tb, tb, 0, st>>>(g, starts, n, offsets, status, a, segs, seg_cap, nseg, err);
    // segments first (the longest work), then the walks that were not split
    if (dist_bits == 16) {
        constexpr int w = TraceWin<uint16_t>::warps;
        k_trace_segs<uint16_t><<<(seg_cap + w - 1) / w, w * 32, 0, st>>>(g, segs, nseg, cells, err);
        k_trace<uint16_t, true><<<(n + w - 1) / w, w * 32, 0, st>>>(g, starts, n, offsets, status, cells,
                                                                    nullptr, nullptr, err, nullptr, kLongWalk);
    } else {
        constexpr int w = TraceWin<uint32_t>::warps;
        k_trace_segs<uint32_t><<<(seg_cap + w - 1) / w, w * 32, 0, st>>>(g, segs, nseg, cells, err);
        const uint32_t *ord = nullptr;
        if (order) {
            count_launch();
            k_order<<<1, 1024, 0, st>>>(offsets, n, order);
            ord = order;
        }
        k_trace<uint32_t, true><<<(n + w - 1) / w, w * 32, 0, st>>>(g, starts, n, offsets, status, cells,
                                                                    nullptr, nullptr, err, ord, kLongWalk);
    }
    return cudaGetLastError();
}

cudaError_t launch_nearest(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                           const int8_t *status, uint32_t *ends, uint32_t *ends_d, cudaStream_t st,
                           uint32_t *err) {
    if (n <= 0) return cudaSuccess;
    if (cudaError_t e = trace_attributes()) return e;
    count_launch();
    if (dist_bits == 16) {
        constexpr int w = TraceWin<uint16_t>::warps;
        k_trace<uint16_t, false><<<(n + w - 1) / w, w * 32, 0, st>>>(g, starts, n, nullptr, status, nullptr,
                                                                     ends, ends_d, err, nullptr);
    } else {
        constexpr int w = TraceWin<uint32_t>::warps;
        k_trace<uint32_t, false><<<(n + w - 1) / w, w * 32, 0, st>>>(g, starts, n, nullptr, status, nullptr,
                                                                     ends, ends_d, err, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_euclid(const GridDev &g, int dist_bits, const uint32_t *starts, int n,
                          uint64_t *offsets, const int8_t *status, uint32_t *cells, bool write,
                          cudaStream_t st, uint32_t *err) {
    if (n <= 0) return cudaSuccess;
    const int nb = (n + kTraceWarps - 1) / kTraceWarps;
    const dim3 tb(kTraceWarps * 32);
    count_launch();
    if (dist_bits == 16) {
        if (write) k_euclid<uint16_t, true><<<nb, tb, 0, st>>>(g, starts, n, offsets, status, cells, err);
        else k_euclid<uint16_t, false><<<nb, tb, 0, st>>>(g, starts, n, offsets, status, cells, err);
    } else {
        if (write) k_euclid<uint32_t, true><<<nb, tb, 0, st>>>(g, starts, n, offsets, status, cells, err);
        else k_euclid<uint32_t, false><<<nb, tb, 0, st>>>(g, starts, n, offsets, status, cells, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_activity(const GridDev &g, int dist_bits, uint32_t L, int32_t *out,
                            cudaStream_t st) {
    const size_t n = (size_t)g.H * g.W;
    count_launch();
    if (dist_bits == 16) k_activity<uint16_t><<<grid_for(n, 256), 256, 0, st>>>(g, L, out);
    else k_activity<uint32_t><<<grid_for(n, 256), 256, 0, st>>>(g, L, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_lengths(const WalkJob *jobs, int njobs, uint32_t *walk_len,
                                 uint64_t *totals, uint32_t *err, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    count_launch();
    k_lengths_batch<<<njobs, 256, 0, st>>>(jobs, walk_len, totals, err);
    return cudaGetLastError();
}

cudaError_t launch_batch_walks(const WalkJob *jobs, int njobs, const uint32_t *walk_len,
                               uint32_t nwalks, uint32_t *order, uint32_t *err, cudaStream_t st) {
    if (njobs <= 0 || nwalks == 0) return cudaSuccess;
    static std::once_flag once;
    static cudaError_t ea = cudaSuccess;
    std::call_once(once, [] {
        ea = cudaFuncSetAttribute((const void *)k_trace_batch, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute((const void *)k_trace_segs_batch,
                                      cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared);
    });
    if (ea != cudaSuccess) return ea;
    count_launch(2);
    k_order_len<<<1, 1024, 0, st>>>(walk_len, nwalks, order);
    k_trace_batch<<<(nwalks + kBatchTraceWarps - 1) / kBatchTraceWarps, kBatchTraceWarps * 32, 0, st>>>(
        jobs, njobs, order, nwalks, err);
    return cudaGetLastError();
}

}  // namespace mpn
