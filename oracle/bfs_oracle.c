/*
 * CPU oracle for BFS levels and closeness sums.  TEST INFRASTRUCTURE ONLY:
 * nothing in the library links or calls this file; only tests, the smoke
 * check and the benchmark's CPU-baseline leg use it.
 *
 * What it computes is the plain definition the method reaches exactly
 * (Eq. 1 and Eq. 2 with the termination rule of §2): level[v] is the hop
 * distance from the source, or -1 when v is unreachable.  It is written as a
 * textbook first-in-first-out queue BFS over the CSR of out-neighbours.  It
 * shares no code with the GPU path.
 *
 * Closeness (§6.2, Eq. 6-7): for every vertex u, far[u] = sum of d(u,v) over
 * the vertices v reachable from u, reach[u] = number of those vertices
 * (u included).  On an undirected graph d(u,v) = d(v,u), so this per-source
 * sum equals the per-target accumulation of Eq. 6.
 *
 * Each BFS is serial; independent sources may run on separate threads.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Serial FIFO BFS.  levels[n] receives the hop distance or -1. */
int or_bfs(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t src, int32_t *levels) {
    if (src < 0 || src >= n) return 1;
    int32_t *queue = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!queue) return 2;
    for (int64_t v = 0; v < n; ++v) levels[v] = -1;
    int64_t head = 0, tail = 0;
    levels[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t v = queue[head++];
        int32_t next_level = levels[v] + 1;
        for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
            int32_t w = col[p];
            if (levels[w] < 0) {
                levels[w] = next_level;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    return 0;
}

typedef struct {
    int64_t n; const int64_t *row_ptr; const int32_t *col;
    int32_t k; const int32_t *srcs; int32_t *levels; /* k*n, source-major */
    int64_t *far; int64_t *reach;                    /* per source (closeness) */
    int32_t *next; int status;
} job_t;

static void *many_worker(void *p) {
    job_t *j = (job_t *)p;
    int32_t *tmp = NULL;
    if (!j->levels) tmp = (int32_t *)malloc((size_t)(j->n > 0 ? j->n : 1) * sizeof(int32_t));
    for (;;) {
        int32_t i = __atomic_fetch_add(j->next, 1, __ATOMIC_RELAXED);
        if (i >= j->k) break;
        int32_t *lv = j->levels ? j->levels + (int64_t)i * j->n : tmp;
        if (or_bfs(j->n, j->row_ptr, j->col, j->srcs[i], lv)) { j->status = 1; continue; }
        if (j->far) {
            int64_t f = 0, r = 0;
            for (int64_t v = 0; v < j->n; ++v)
                if (lv[v] >= 0) { f += lv[v]; r += 1; }
            j->far[i] = f;
            j->reach[i] = r;
        }
    }
    free(tmp);
    return NULL;
}

static int run_many(job_t *proto, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int32_t next = 0;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) { jobs[t] = *proto; jobs[t].next = &next; jobs[t].status = 0; }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, many_worker, &jobs[t]);
    many_worker(&jobs[0]);
    int st = jobs[0].status;
    for (int t = 1; t < nthreads; ++t) { pthread_join(th[t], NULL); st |= jobs[t].status; }
    return st;
}

/* k independent serial BFSs; levels is k*n, levels[c*n + v]. */
int or_bfs_many(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t k, const int32_t *srcs,
                int32_t *levels, int nthreads) {
    job_t j;
    memset(&j, 0, sizeof j);
    j.n = n; j.row_ptr = row_ptr; j.col = col; j.k = k; j.srcs = srcs; j.levels = levels;
    return run_many(&j, nthreads);
}

/* Distance sums from each listed vertex: far[i] = sum_v d(verts[i], v),
 * reach[i] = |{v reachable}|.  With verts = all vertices this is the full
 * closeness input. */
int or_far_reach(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t k, const int32_t *verts,
                 int64_t *far, int64_t *reach, int nthreads) {
    job_t j;
    memset(&j, 0, sizeof j);
    j.n = n; j.row_ptr = row_ptr; j.col = col; j.k = k; j.srcs = verts; j.levels = NULL;
    j.far = far; j.reach = reach;
    return run_many(&j, nthreads);
}
