/*
 * Seeded synthetic workload generators (obstacle grids, mazes, end-points).
 *
 * This module produces inputs only. It holds none of the path planner's
 * arithmetic (no propagation, no distances, no tracing), so both the CUDA
 * path and the CPU oracle may consume what it writes.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * SplitMix64 (Steele, Lea & Flood, 2014), both written here from their
 * published definitions. All arithmetic is 64-bit unsigned, so the streams are
 * identical on x86-64 and AArch64.
 *
 * Mask convention everywhere: row-major H x W uint8, nonzero = obstacle.
 * A linear cell index is y * W + x.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* Uniform integer in [0, n) by the multiply-high method (n >= 1). */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

/* Uniform integer in [lo, hi] inclusive. */
static inline int64_t rng_range(rng_t *r, int64_t lo, int64_t hi) {
    return lo + (int64_t)rng_below(r, (uint64_t)(hi - lo + 1));
}

/* ---- exported helpers ------------------------------------------------- */

/* Derive an independent sub-seed from (seed, stream) so that each generator
 * stage of a workload draws from its own stream. */
uint64_t synth_subseed(uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ULL);
    splitmix64_next(&x);
    return splitmix64_next(&x);
}

/* First n outputs of the generator for `seed` (used by tests to pin the
 * stream against the published reference values). */
void synth_rng_stream(uint64_t seed, uint64_t *out, int64_t n) {
    rng_t r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = rng_next(&r);
}

/* Raw xoshiro256** stream from an explicit 256-bit state (tests compare it
 * with the reference implementation's published first outputs). */
void synth_xoshiro_from_state(const uint64_t state[4], uint64_t *out, int64_t n) {
    rng_t r;
    memcpy(r.s, state, sizeof r.s);
    for (int64_t i = 0; i < n; ++i) out[i] = rng_next(&r);
}

void synth_splitmix_stream(uint64_t seed, uint64_t *out, int64_t n) {
    uint64_t x = seed;
    for (int64_t i = 0; i < n; ++i) out[i] = splitmix64_next(&x);
}

/* Uniform integers in [lo, hi] (used by the batched workload for sizes and
 * end-point counts, and by the serving driver for Poisson arrival gaps). */
void synth_uniform_ints(uint64_t seed, int64_t lo, int64_t hi, int64_t *out, int64_t n) {
    rng_t r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = rng_range(&r, lo, hi);
}

/* Uniform doubles in [0, 1) with 53 random bits. */
void synth_uniform_doubles(uint64_t seed, double *out, int64_t n) {
    rng_t r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = (double)(rng_next(&r) >> 11) * (1.0 / 9007199254740992.0);
}

/* Each cell an obstacle independently with probability p. */
void synth_bernoulli(uint8_t *mask, int64_t H, int64_t W, double p, uint64_t seed) {
    rng_t r;
    rng_seed(&r, seed);
    /* compare 53-bit uniforms against a 53-bit threshold: exact and portable */
    const uint64_t thr = (uint64_t)(p * 9007199254740992.0);
    const int64_t n = H * W;
    for (int64_t i = 0; i < n; ++i) mask[i] = (uint8_t)((rng_next(&r) >> 11) < thr);
}

void synth_fill(uint8_t *mask, int64_t n, uint8_t v) { memset(mask, v, (size_t)n); }

/*
 * Perfect maze by randomized depth-first search (iterative, explicit stack).
 * Lattice cells sit at pixels (2i, 2j) with 2i < H and 2j < W. Every pixel
 * starts as wall; lattice cells are opened, and the wall pixel between two
 * lattice cells is opened when the search moves between them. The search
 * starts at lattice cell (0, 0) and, at each step, moves to a uniformly chosen
 * unvisited lattice neighbour (4-neighbourhood), backtracking when there is
 * none. Returns 0, or -1 if memory runs out.
 */
int synth_dfs_maze(uint8_t *mask, int64_t H, int64_t W, uint64_t seed) {
    const int64_t LH = (H + 1) / 2, LW = (W + 1) / 2, LN = LH * LW;
    memset(mask, 1, (size_t)(H * W));
    if (LN <= 0) return 0;
    uint8_t *seen = (uint8_t *)calloc((size_t)LN, 1);
    int64_t *stack = (int64_t *)malloc((size_t)LN * sizeof(int64_t));
    if (!seen || !stack) { free(seen); free(stack); return -1; }
    rng_t r;
    rng_seed(&r, seed);
    static const int dI[4] = {-1, 0, 1, 0};
    static const int dJ[4] = {0, 1, 0, -1};
    int64_t top = 0;
    stack[top++] = 0;
    seen[0] = 1;
    mask[0] = 0;
    while (top > 0) {
        const int64_t c = stack[top - 1];
        const int64_t ci = c / LW, cj = c % LW;
        int64_t cand[4];
        int nc = 0;
        for (int k = 0; k < 4; ++k) {
            const int64_t ni = ci + dI[k], nj = cj + dJ[k];
            if (ni < 0 || nj < 0 || ni >= LH || nj >= LW) continue;
            if (!seen[ni * LW + nj]) cand[nc++] = ni * LW + nj;
        }
        if (nc == 0) { --top; continue; }
        const int64_t nx = cand[rng_below(&r, (uint64_t)nc)];
        const int64_t ni = nx / LW, nj = nx % LW;
        seen[nx] = 1;
        mask[(2 * ni) * W + 2 * nj] = 0;              /* open the lattice cell */
        mask[(ci + ni) * W + (cj + nj)] = 0;          /* open the wall between (pixel midpoint) */
        stack[top++] = nx;
    }
    free(seen);
    free(stack);
    return 0;
}

/*
 * Open a fraction of the wall pixels that still separate two lattice cells of
 * a maze made by synth_dfs_maze: candidates are pixels (2i+1, 2j) with both
 * (2i, 2j) and (2i+2, 2j) inside the grid, and (2i, 2j+1) with both (2i, 2j)
 * and (2i, 2j+2) inside, that are still walls. floor(frac * count) of them are
 * chosen uniformly without replacement (partial Fisher-Yates) and opened.
 * Returns the number opened, or -1 if memory runs out.
 */
int64_t synth_remove_walls(uint8_t *mask, int64_t H, int64_t W, double frac, uint64_t seed) {
    int64_t cap = 0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            const int vwall = (y % 2 == 1) && (x % 2 == 0) && (y + 1 < H);
            const int hwall = (y % 2 == 0) && (x % 2 == 1) && (x + 1 < W);
            if ((vwall || hwall) && mask[y * W + x]) ++cap;
        }
    if (cap == 0) return 0;
    int64_t *idx = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!idx) return -1;
    int64_t n = 0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            const int vwall = (y % 2 == 1) && (x % 2 == 0) && (y + 1 < H);
            const int hwall = (y % 2 == 0) && (x % 2 == 1) && (x + 1 < W);
            if ((vwall || hwall) && mask[y * W + x]) idx[n++] = y * W + x;
        }
    const int64_t k = (int64_t)(frac * (double)n);
    rng_t r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < k; ++i) {
        const int64_t j = i + (int64_t)rng_below(&r, (uint64_t)(n - i));
        const int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
        mask[idx[i]] = 0;
    }
    free(idx);
    return k;
}

/*
 * Axis-aligned obstacle rectangles with heights and widths uniform in
 * [smin, smax] (clipped to the grid) and top-left corners uniform over the
 * positions where they fit, added until their union covers at least
 * cover_frac of the grid. Returns the number of rectangles, or -1 if memory
 * runs out.
 */
int64_t synth_rectangles(uint8_t *mask, int64_t H, int64_t W, int64_t smin, int64_t smax,
                         double cover_frac, uint64_t seed) {
    const int64_t n = H * W;
    uint8_t *cov = (uint8_t *)calloc((size_t)n, 1);
    if (!cov) return -1;
    rng_t r;
    rng_seed(&r, seed);
    const int64_t need = (int64_t)(cover_frac * (double)n + 0.999999);
    int64_t covered = 0, nrect = 0;
    while (covered < need) {
        int64_t h = rng_range(&r, smin, smax), w = rng_range(&r, smin, smax);
        if (h > H) h = H;
        if (w > W) w = W;
        const int64_t y0 = rng_range(&r, 0, H - h), x0 = rng_range(&r, 0, W - w);
        for (int64_t y = y0; y < y0 + h; ++y) {
            uint8_t *cr = cov + y * W, *mr = mask + y * W;
            for (int64_t x = x0; x < x0 + w; ++x) {
                covered += !cr[x];
                cr[x] = 1;
                mr[x] = 1;
            }
        }
        ++nrect;
    }
    free(cov);
    return nrect;
}

/*
 * k distinct free cells, uniform without replacement, as linear indices in
 * draw order. Sparse case (k small next to the free count): rejection sampling
 * over all cells with a duplicate check. Dense case: enumerate the free cells
 * and take a partial Fisher-Yates shuffle. Returns k, or -1 if there are fewer
 * than k free cells or memory runs out.
 */
int64_t synth_sample_free(const uint8_t *mask, int64_t H, int64_t W, int64_t k, uint64_t seed,
                          uint32_t *out) {
    const int64_t n = H * W;
    int64_t nfree = 0;
    for (int64_t i = 0; i < n; ++i) nfree += !mask[i];
    if (nfree < k) return -1;
    if (k == 0) return 0;
    rng_t r;
    rng_seed(&r, seed);
    if (k * 8 <= nfree) {
        int64_t got = 0;
        while (got < k) {
            const int64_t c = (int64_t)rng_below(&r, (uint64_t)n);
            if (mask[c]) continue;
            int dup = 0;
            for (int64_t i = 0; i < got && !dup; ++i) dup = ((int64_t)out[i] == c);
            if (dup) continue;
            out[got++] = (uint32_t)c;
        }
        return k;
    }
    int64_t *cells = (int64_t *)malloc((size_t)nfree * sizeof(int64_t));
    if (!cells) return -1;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (!mask[i]) cells[m++] = i;
    for (int64_t i = 0; i < k; ++i) {
        const int64_t j = i + (int64_t)rng_below(&r, (uint64_t)(m - i));
        const int64_t t = cells[i]; cells[i] = cells[j]; cells[j] = t;
        out[i] = (uint32_t)cells[i];
    }
    free(cells);
    return k;
}
