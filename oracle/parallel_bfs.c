/*
 * Parallel CPU baseline -- TEST AND BENCHMARK INFRASTRUCTURE ONLY, not the
 * oracle. A level-synchronous multi-source BFS on all host cores (OpenMP):
 * every cell of the current level's frontier claims its free, unvisited
 * 8-neighbours with a compare-and-swap on the distance (INF -> level + 1) and
 * appends them to a thread-local buffer; the buffers are concatenated into the
 * next frontier. The distance of a cell is the level at which it is first
 * claimed, which does not depend on which thread claims it, so the result is
 * the unique hop distance of the layer recurrence (Methods, "Activity Map
 * Generation") -- the same value oracle_bfs computes serially; the tests check
 * the two against each other. Status codes as in oracle.c: 0 ok, 1 invalid
 * argument, 2 out of memory, 6 target on an obstacle.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PB_INF 0xFFFFFFFFu

typedef struct {
    uint32_t *a;
    int64_t n, cap;
} buf_t;

static int push(buf_t *b, uint32_t v) {
    if (b->n == b->cap) {
        const int64_t cap = b->cap ? 2 * b->cap : 4096;
        uint32_t *a = (uint32_t *)realloc(b->a, (size_t)cap * sizeof(uint32_t));
        if (!a) return 0;
        b->a = a;
        b->cap = cap;
    }
    b->a[b->n++] = v;
    return 1;
}

int parallel_bfs(const uint8_t *mask, int64_t H, int64_t W, const uint32_t *targets, int64_t nt,
                 uint32_t *dist, uint32_t *layers_out, int32_t *threads_out) {
    if (!mask || !dist || !targets || H < 1 || W < 1 || nt < 1) return 1;
    const int64_t N = H * W;
    for (int64_t i = 0; i < nt; ++i) {
        if ((int64_t)targets[i] >= N) return 1;
        if (mask[targets[i]]) return 6;
    }
    uint32_t *cur = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    uint32_t *nxt = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return 2;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) dist[i] = PB_INF;
    int64_t ncur = 0;
    for (int64_t i = 0; i < nt; ++i)
        if (dist[targets[i]] == PB_INF) {
            dist[targets[i]] = 0;
            cur[ncur++] = targets[i];
        }
    int threads = 1;
    int failed = 0;
    uint32_t level = 0;
    while (ncur > 0 && !failed) {
        int64_t nnext = 0;
#pragma omp parallel
        {
#pragma omp single
            threads = omp_get_num_threads();
            buf_t local = {0, 0, 0};
#pragma omp for schedule(dynamic, 1024)
            for (int64_t i = 0; i < ncur; ++i) {
                const int64_t c = cur[i], y = c / W, x = c % W;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int64_t yy = y + dy, xx = x + dx;
                        if ((!dy && !dx) || yy < 0 || xx < 0 || yy >= H || xx >= W) continue;
                        const int64_t n = yy * W + xx;
                        if (mask[n]) continue;
                        uint32_t expect = PB_INF;
                        if (__atomic_load_n(&dist[n], __ATOMIC_RELAXED) == PB_INF &&
                            __atomic_compare_exchange_n(&dist[n], &expect, level + 1, 0,
                                                        __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
                            if (!push(&local, (uint32_t)n)) {
#pragma omp atomic write
                                failed = 1;
                            }
                        }
                    }
            }
            int64_t at;
#pragma omp atomic capture
            {
                at = nnext;
                nnext += local.n;
            }
            if (local.n) memcpy(nxt + at, local.a, (size_t)local.n * sizeof(uint32_t));
            free(local.a);
        }
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
        ncur = nnext;
        if (ncur) ++level;
    }
    free(cur);
    free(nxt);
    if (failed) return 2;
    if (layers_out) *layers_out = level;
    if (threads_out) *threads_out = threads;
    return 0;
}
