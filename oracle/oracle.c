/*
 * CPU ORACLE for the max-pooling path planner (oMAP, arXiv 2004.00540).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code. The product path (the CUDA
 * library) never calls it, and the two share no code.
 *
 * What the method computes. Methods, "Activity Map Generation": each layer is
 *     A_l = ReLU( maxpool3x3(A_{l-1}) + I_e + I_s ),   A_0 = I_s,
 * with zero padding, I_e = -maxint on obstacles and 0 elsewhere (Methods,
 * "Input"), I_s = 1 on sources. By induction on l, A_l(c) = l + 1 - d(c) when
 * the 8-connected unit-cost hop distance d(c) from the nearest source is at
 * most l, and 0 otherwise (sources read l + 1, their free neighbours after the
 * first layer read 1). So the layer at which a cell first turns positive is
 * d(c), the plain multi-source breadth-first-search distance, and following the
 * maximum neighbour back (Methods, "Path Reconstruction") means stepping to a
 * neighbour with distance d - 1.
 *
 * The oracle therefore computes:
 *   oracle_bfs    - that plain definition: FIFO multi-source BFS over free
 *                   cells, 8 neighbours, unit cost (Results, "oMAP versus
 *                   Dijkstra": all moves cost 1). A fixed depth L leaves cells
 *                   with d > L unreached, like a network of L layers.
 *   oracle_trace  - simple path reconstruction from each start: repeatedly
 *                   step to an 8-neighbour with distance d - 1 until d = 0.
 *                   The paper breaks ties at random; this oracle takes the
 *                   first such neighbour in the order (dy,dx) = (-1,-1),
 *                   (-1,0), (-1,1), (0,-1), (0,1), (1,-1), (1,0), (1,1), which
 *                   is the lowest linear index.
 *   oracle_omap   - the layer recurrence written out literally with int32
 *                   arrays, used only to pin the relation above on small grids.
 *   oracle_euclid_trace - Euclidean path reconstruction (Eq. 1 and the
 *                   straightening rule that follows it).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - stop rule: the first layer that activates no new cell (the paper's "no
 *     zero left except at obstacles" never holds with unreachable pockets);
 *     unreachable cells keep the sentinel 0xFFFFFFFF;
 *   - diagonal moves between two corner-touching obstacles are allowed (a 3x3
 *     max pool passes activity there);
 *   - outside the grid nothing is traversable (zero padding);
 *   - a target on an obstacle is an error, a target may equal a start.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_EOBSTACLE 6
#define OR_INF 0xFFFFFFFFu

static const int DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
static const int DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};

static int validate(int64_t H, int64_t W, const uint32_t *idx, int64_t n, int need_one) {
    if (H < 1 || W < 1 || H * W >= (int64_t)OR_INF) return OR_EINVAL;
    if (n < 0 || (need_one && n < 1)) return OR_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if ((int64_t)idx[i] >= H * W) return OR_EINVAL;
    return OR_OK;
}

/*
 * Multi-source BFS distances. dist: H*W uint32, OR_INF where unreached or on
 * an obstacle. max_layers = 0 runs to convergence; L > 0 stops after layer L.
 * *layers_out = the largest finite distance (the number of layers the network
 * needs, Methods, "Determining the number of layers L").
 */
int oracle_bfs(const uint8_t *mask, int64_t H, int64_t W, const uint32_t *targets, int64_t nt,
               uint32_t max_layers, uint32_t *dist, uint32_t *layers_out) {
    int st = validate(H, W, targets, nt, 1);
    if (st) return st;
    for (int64_t i = 0; i < nt; ++i)
        if (mask[targets[i]]) return OR_EOBSTACLE;
    const int64_t N = H * W;
    uint32_t *queue = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    if (!queue) return OR_ENOMEM;
    for (int64_t i = 0; i < N; ++i) dist[i] = OR_INF;
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < nt; ++i) {
        const uint32_t t = targets[i];
        if (dist[t] == OR_INF) {
            dist[t] = 0;
            queue[tail++] = t;
        }
    }
    uint32_t maxd = 0;
    while (head < tail) {
        const uint32_t c = queue[head++];
        const uint32_t d = dist[c];
        if (d > maxd) maxd = d;
        if (max_layers && d >= max_layers) continue;
        const int64_t y = c / W, x = c % W;
        for (int k = 0; k < 8; ++k) {
            const int64_t ny = y + DY[k], nx = x + DX[k];
            if (ny < 0 || nx < 0 || ny >= H || nx >= W) continue;
            const int64_t n = ny * W + nx;
            if (mask[n] || dist[n] != OR_INF) continue;
            dist[n] = d + 1;
            queue[tail++] = (uint32_t)n;
        }
    }
    free(queue);
    if (layers_out) *layers_out = maxd;
    return OR_OK;
}

/*
 * Simple path reconstruction. offsets: ns + 1 entries, offsets[0] = 0 and
 * offsets[i+1] - offsets[i] = d(start_i) + 1 for a reachable start, else 0.
 * cells: the concatenated paths, start first, target last. status per start:
 * 0 ok, 1 unreachable, 2 start on an obstacle. If the total exceeds cap the
 * offsets are still filled and OR_ENOMEM is returned.
 */
int oracle_trace(const uint8_t *mask, const uint32_t *dist, int64_t H, int64_t W,
                 const uint32_t *starts, int64_t ns, uint64_t *offsets, uint32_t *cells,
                 uint64_t cap, int8_t *status) {
    int st = validate(H, W, starts, ns, 0);
    if (st) return st;
    offsets[0] = 0;
    for (int64_t i = 0; i < ns; ++i) {
        const uint32_t s = starts[i];
        uint64_t len = 0;
        if (mask[s]) status[i] = 2;
        else if (dist[s] == OR_INF) status[i] = 1;
        else { status[i] = 0; len = (uint64_t)dist[s] + 1; }
        offsets[i + 1] = offsets[i] + len;
    }
    if (offsets[ns] > cap) return OR_ENOMEM;
    for (int64_t i = 0; i < ns; ++i) {
        if (status[i] != 0) continue;
        uint64_t o = offsets[i];
        int64_t c = starts[i];
        cells[o++] = (uint32_t)c;
        while (dist[c] > 0) {
            const uint32_t want = dist[c] - 1;
            const int64_t y = c / W, x = c % W;
            int64_t next = -1;
            for (int k = 0; k < 8 && next < 0; ++k) {
                const int64_t ny = y + DY[k], nx = x + DX[k];
                if (ny < 0 || nx < 0 || ny >= H || nx >= W) continue;
                const int64_t n = ny * W + nx;
                if (!mask[n] && dist[n] == want) next = n;
            }
            if (next < 0) return OR_EINVAL; /* not a BFS distance plane */
            c = next;
            cells[o++] = (uint32_t)c;
        }
    }
    return OR_OK;
}

/*
 * The layer recurrence written out, L layers, int32 activity (Methods,
 * "Activity Map Generation"): A_0 = I_s; A_l = max(0, maxpool3x3(A_{l-1}) +
 * I_e + I_s) with zero padding and I_e = -maxint = -(2^31 - 1) on obstacles.
 * A: H*W int32 output (the final activity map O). Grids up to 256 x 256.
 */
int oracle_omap(const uint8_t *mask, int64_t H, int64_t W, const uint32_t *targets, int64_t nt,
                int32_t L, int32_t *A) {
    int st = validate(H, W, targets, nt, 1);
    if (st) return st;
    if (H * W > 256 * 256 || L < 0) return OR_EINVAL;
    const int64_t N = H * W;
    const int64_t maxint = 2147483647;
    int32_t *Ie = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *Is = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    int32_t *prev = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!Ie || !Is || !prev) { free(Ie); free(Is); free(prev); return OR_ENOMEM; }
    for (int64_t i = 0; i < N; ++i) Ie[i] = mask[i] ? (int32_t)(-maxint) : 0;
    for (int64_t i = 0; i < nt; ++i) Is[targets[i]] = 1;
    memcpy(A, Is, (size_t)N * sizeof(int32_t));
    for (int32_t l = 1; l <= L; ++l) {
        memcpy(prev, A, (size_t)N * sizeof(int32_t));
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int64_t m = 0; /* zero padding: the pad value 0 enters the max */
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int64_t yy = y + dy, xx = x + dx;
                        const int64_t v = (yy < 0 || xx < 0 || yy >= H || xx >= W)
                                              ? 0 : prev[yy * W + xx];
                        if (v > m) m = v;
                    }
                const int64_t s = m + Ie[y * W + x] + Is[y * W + x];
                A[y * W + x] = (int32_t)(s > 0 ? s : 0);
            }
    }
    free(Ie); free(Is); free(prev);
    return OR_OK;
}

/*
 * Euclidean path reconstruction (Methods, "Path Reconstruction", Eq. 1):
 * from the start, step to the 4-neighbour (left, right, up, down) with the
 * largest activity, i.e. the smallest distance, until a source (d = 0) is
 * reached; then drop interior points P(t) whose neighbours on the path are
 * exactly sqrt(2) apart.
 *
 * Readings (Eq. 1 leaves plateaus undefined): ties among 4-neighbours go to
 * the first of (0,-1), (0,1), (-1,0), (1,0), the order Eq. 1 lists them
 * (O(i,j-1), O(i,j+1), O(i-1,j), O(i+1,j), i = row). If no 4-neighbour has
 * distance d - 1, the nearest cell with d - 1 is diagonal; the walk then steps
 * to the first 4-neighbour with distance d that is itself 4-adjacent to a cell
 * with distance d - 1 (the corner of that diagonal move), and if both corners
 * are obstacles it takes the diagonal step to the first 8-neighbour with
 * d - 1 in the simple-reconstruction order. Every two steps lower d by one, so
 * the walk ends. The straightening rule compares P(t+1) with the previous
 * point of the path as straightened so far (a forward scan), so every removal
 * replaces two axis-aligned steps by one diagonal step and the result stays
 * 8-connected.
 *
 * Output like oracle_trace, with offsets[i+1] - offsets[i] the straightened
 * length. OR_ENOMEM if cap is too small (offsets valid up to that start).
 */
static int64_t euclid_next(const uint8_t *mask, const uint32_t *dist, int64_t H, int64_t W,
                           int64_t c) {
    static const int EY[4] = {0, 0, -1, 1};
    static const int EX[4] = {-1, 1, 0, 0};
    const uint32_t d = dist[c];
    const int64_t y = c / W, x = c % W;
    for (int q = 0; q < 4; ++q) {            /* a 4-neighbour one step closer */
        const int64_t ny = y + EY[q], nx = x + EX[q];
        if (ny < 0 || nx < 0 || ny >= H || nx >= W) continue;
        const int64_t n = ny * W + nx;
        if (!mask[n] && dist[n] == d - 1) return n;
    }
    for (int q = 0; q < 4; ++q) {            /* corner of a diagonal move */
        const int64_t ny = y + EY[q], nx = x + EX[q];
        if (ny < 0 || nx < 0 || ny >= H || nx >= W) continue;
        const int64_t n = ny * W + nx;
        if (mask[n] || dist[n] != d) continue;
        for (int r = 0; r < 4; ++r) {
            const int64_t my = ny + EY[r], mx = nx + EX[r];
            if (my < 0 || mx < 0 || my >= H || mx >= W) continue;
            const int64_t m = my * W + mx;
            if (!mask[m] && dist[m] == d - 1) return n;
        }
    }
    for (int k = 0; k < 8; ++k) {            /* squeeze between two obstacles */
        const int64_t ny = y + DY[k], nx = x + DX[k];
        if (ny < 0 || nx < 0 || ny >= H || nx >= W) continue;
        const int64_t n = ny * W + nx;
        if (!mask[n] && dist[n] == d - 1) return n;
    }
    return -1;
}

int oracle_euclid_trace(const uint8_t *mask, const uint32_t *dist, int64_t H, int64_t W,
                        const uint32_t *starts, int64_t ns, uint64_t *offsets, uint32_t *cells,
                        uint64_t cap, int8_t *status) {
    int st = validate(H, W, starts, ns, 0);
    if (st) return st;
    offsets[0] = 0;
    uint32_t *raw = NULL;
    int64_t rawcap = 0;
    for (int64_t i = 0; i < ns; ++i) {
        const uint32_t s = starts[i];
        uint64_t o = offsets[i];
        if (mask[s]) { status[i] = 2; offsets[i + 1] = o; continue; }
        if (dist[s] == OR_INF) { status[i] = 1; offsets[i + 1] = o; continue; }
        const int64_t need = 2 * (int64_t)dist[s] + 1;
        if (need > rawcap) {
            uint32_t *nr = (uint32_t *)realloc(raw, (size_t)need * sizeof(uint32_t));
            if (!nr) { free(raw); return OR_ENOMEM; }
            raw = nr;
            rawcap = need;
        }
        int64_t k = 0, c = s;
        raw[k++] = (uint32_t)c;
        status[i] = 0;
        while (dist[c] > 0) {
            c = euclid_next(mask, dist, H, W, c);
            if (c < 0) { free(raw); return OR_EINVAL; } /* not a BFS distance plane */
            raw[k++] = (uint32_t)c;
        }
        /* straighten, scanning forward: P(t) is dropped when the last kept
         * point and P(t+1) are exactly sqrt(2) apart, so each dropped point
         * turns two axis steps into one diagonal step */
        int64_t last = -1;
        for (int64_t t = 0; t < k; ++t) {
            int keep = 1;
            if (t > 0 && t < k - 1) {
                const int64_t ay = raw[last] / W, ax = raw[last] % W;
                const int64_t by = raw[t + 1] / W, bx = raw[t + 1] % W;
                const int64_t dy = ay - by, dx = ax - bx;
                if (dy * dy + dx * dx == 2) keep = 0;
            }
            if (keep) {
                if (o >= cap) { free(raw); offsets[i + 1] = o; return OR_ENOMEM; }
                cells[o++] = raw[t];
                last = t;
            }
        }
        offsets[i + 1] = o;
    }
    free(raw);
    return OR_OK;
}
