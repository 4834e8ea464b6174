/*
 * Seeded synthetic graph generators: the inputs for every test, parity check
 * and benchmark.  This file holds no BFS arithmetic; it only produces CSR
 * graphs and source lists, and is shared by the CPU oracle and the GPU path.
 *
 * Randomness: every random draw is a pure function of (seed, stream, index),
 * computed with the splitmix64 finaliser (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014).  Results are
 * therefore identical for any thread count and on any host (x86_64, aarch64):
 * integer arithmetic only, except the RMAT/ER probability thresholds, which
 * are converted to integers once.
 *
 * Generators:
 *   RMAT        Graph500-style recursive quadrant choice, vertex labels
 *               scrambled by a seeded bijection on [0, 2^scale).
 *   grid        rows x cols 4-neighbour grid, a seeded fraction of edges
 *               deleted, a fraction of uniform random shortcuts added.
 *   BA          Barabasi-Albert preferential attachment by the linear-time
 *               method of Batagelj & Brandes ("Efficient generation of large
 *               random networks", Phys. Rev. E 71, 2005).
 *   RGG         2D random geometric graph in the unit square, integer
 *               coordinates on a 2^31 lattice, radius from the target
 *               average degree.
 * All graphs are returned as CSR (int64 row_ptr, int32 col), rows sorted,
 * self loops and duplicate arcs removed; undirected graphs are symmetric.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct gg_graph {
    int64_t n;
    int64_t nnz;
    int64_t *row_ptr; /* n+1 */
    int32_t *col;     /* nnz */
} gg_graph;

typedef struct gg_batch {
    int32_t g;
    int64_t total_n;
    int64_t total_nnz;
    int64_t *vtx_off;  /* g+1 */
    int64_t *edge_off; /* g+1 */
    int64_t *row_ptr;  /* total_n + g : per graph n_i+1 entries, local to the graph's edge block */
    int32_t *col;      /* total_nnz, local vertex ids */
} gg_batch;

/* ------------------------------------------------------------------ RNG */
static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t rng(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t k = mix64(seed * 0x9E3779B97F4A7C15ULL + stream * 0xD1B54A32D192ED03ULL + 0x2545F4914F6CDD1DULL);
    return mix64(k + (i + 1) * 0x9E3779B97F4A7C15ULL);
}
/* unbiased-enough map of a 64-bit draw onto [0, n) (multiply-high) */
static inline uint64_t bounded(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

uint64_t gg_rng(uint64_t seed, uint64_t stream, uint64_t i) { return rng(seed, stream, i); }

enum { S_RMAT = 1, S_SCRAMBLE = 2, S_GRID_DEL = 3, S_GRID_SC = 4, S_BA = 5, S_RGG = 6,
       S_SRC = 7, S_BATCH = 8, S_ER = 9 };

/* ------------------------------------------------------- parallel helper */
typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi, int tid);
typedef struct { range_fn fn; void *ctx; int64_t n, chunk; int64_t *next; int tid; } pf_arg;

static void *pf_worker(void *p) {
    pf_arg *a = (pf_arg *)p;
    for (;;) {
        int64_t lo = __atomic_fetch_add(a->next, a->chunk, __ATOMIC_RELAXED);
        if (lo >= a->n) break;
        int64_t hi = lo + a->chunk < a->n ? lo + a->chunk : a->n;
        a->fn(a->ctx, lo, hi, a->tid);
    }
    return NULL;
}
/* dynamic-chunked parallel for over [0, n) */
static void parallel_for(int64_t n, int64_t chunk, int nthreads, range_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (chunk < 1) chunk = 1;
    int64_t next = 0;
    pthread_t th[256];
    pf_arg args[256];
    for (int t = 0; t < nthreads; ++t) {
        args[t].fn = fn; args[t].ctx = ctx; args[t].n = n; args[t].chunk = chunk;
        args[t].next = &next; args[t].tid = t;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, pf_worker, &args[t]);
    pf_worker(&args[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------ CSR build */
typedef struct {
    int64_t n, ne;
    const int32_t *u, *v;
    int symmetrize;
    int64_t *cnt;     /* n+1 */
    int64_t *cursor;  /* n */
    int32_t *tmp;
    int64_t *ucnt;    /* unique count per row */
    int64_t *row_ptr;
    int32_t *col;
} csr_ctx;

static void csr_count(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    csr_ctx *c = (csr_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        int32_t a = c->u[e], b = c->v[e];
        if (a == b) continue;
        __atomic_fetch_add(&c->cnt[a], 1, __ATOMIC_RELAXED);
        if (c->symmetrize) __atomic_fetch_add(&c->cnt[b], 1, __ATOMIC_RELAXED);
    }
}
static void csr_fill(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    csr_ctx *c = (csr_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        int32_t a = c->u[e], b = c->v[e];
        if (a == b) continue;
        int64_t pa = __atomic_fetch_add(&c->cursor[a], 1, __ATOMIC_RELAXED);
        c->tmp[pa] = b;
        if (c->symmetrize) {
            int64_t pb = __atomic_fetch_add(&c->cursor[b], 1, __ATOMIC_RELAXED);
            c->tmp[pb] = a;
        }
    }
}
static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}
static void csr_sort(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    csr_ctx *c = (csr_ctx *)p;
    for (int64_t r = lo; r < hi; ++r) {
        int64_t b = c->cnt[r], e = c->cnt[r + 1];
        int64_t len = e - b;
        int32_t *row = c->tmp + b;
        if (len > 1) {
            if (len <= 16) { /* insertion sort for short rows */
                for (int64_t i = 1; i < len; ++i) {
                    int32_t x = row[i]; int64_t j = i - 1;
                    while (j >= 0 && row[j] > x) { row[j + 1] = row[j]; --j; }
                    row[j + 1] = x;
                }
            } else {
                qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
            }
        }
        int64_t k = 0;
        for (int64_t i = 0; i < len; ++i)
            if (k == 0 || row[i] != row[k - 1]) row[k++] = row[i];
        c->ucnt[r] = k;
    }
}
static void csr_compact(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    csr_ctx *c = (csr_ctx *)p;
    for (int64_t r = lo; r < hi; ++r)
        memcpy(c->col + c->row_ptr[r], c->tmp + c->cnt[r], (size_t)c->ucnt[r] * sizeof(int32_t));
}

/* Build a CSR from an edge list.  symmetrize=1: both directions are added. */
gg_graph *gg_from_edges(int64_t n, int64_t ne, const int32_t *u, const int32_t *v, int symmetrize,
                        int nthreads) {
    csr_ctx c;
    memset(&c, 0, sizeof c);
    c.n = n; c.ne = ne; c.u = u; c.v = v; c.symmetrize = symmetrize;
    c.cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    c.cursor = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    c.ucnt = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!c.cnt || !c.cursor || !c.ucnt || !g) return NULL;
    parallel_for(ne, 1 << 16, nthreads, csr_count, &c);
    /* exclusive scan of counts -> cnt becomes row starts (n+1 entries) */
    int64_t run = 0;
    for (int64_t i = 0; i < n; ++i) { int64_t d = c.cnt[i]; c.cnt[i] = run; run += d; }
    c.cnt[n] = run;
    memcpy(c.cursor, c.cnt, (size_t)n * sizeof(int64_t));
    c.tmp = (int32_t *)malloc((size_t)(run > 0 ? run : 1) * sizeof(int32_t));
    if (!c.tmp) return NULL;
    parallel_for(ne, 1 << 16, nthreads, csr_fill, &c);
    parallel_for(n, 4096, nthreads, csr_sort, &c);
    g->n = n;
    g->row_ptr = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) { g->row_ptr[i] = acc; acc += c.ucnt[i]; }
    g->row_ptr[n] = acc;
    g->nnz = acc;
    g->col = (int32_t *)malloc((size_t)(acc > 0 ? acc : 1) * sizeof(int32_t));
    c.row_ptr = g->row_ptr; c.col = g->col;
    parallel_for(n, 4096, nthreads, csr_compact, &c);
    free(c.cnt); free(c.cursor); free(c.ucnt); free(c.tmp);
    return g;
}

void gg_free(gg_graph *g) {
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g);
}
int64_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_nnz(const gg_graph *g) { return g->nnz; }
void gg_copy(const gg_graph *g, int64_t *row_ptr, int32_t *col) {
    memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
}

/* ----------------------------------------------------------------- RMAT */
typedef struct {
    int scale; uint64_t seed; uint32_t ta, tab, tabc; int scramble;
    int32_t *u, *v; uint64_t sm[8]; /* scramble multipliers/addends */
} rmat_ctx;

static inline uint32_t scramble_id(const rmat_ctx *c, uint32_t x) {
    uint64_t mask = (c->scale >= 32) ? 0xFFFFFFFFULL : ((1ULL << c->scale) - 1ULL);
    int s = c->scale / 2 + 1;
    uint64_t y = x;
    for (int r = 0; r < 4; ++r) {
        y = (y * (c->sm[2 * r] | 1ULL) + c->sm[2 * r + 1]) & mask; /* odd multiply: bijection mod 2^k */
        y ^= (y >> s);                                              /* xorshift: bijection on k bits */
    }
    return (uint32_t)y;
}

static void rmat_gen(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    rmat_ctx *c = (rmat_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint32_t a = 0, b = 0;
        for (int d = 0; d < c->scale; d += 2) {
            uint64_t r = rng(c->seed, S_RMAT, (uint64_t)e * 32 + (uint64_t)d);
            for (int h = 0; h < 2 && d + h < c->scale; ++h) {
                uint32_t x = (uint32_t)(h ? (r >> 32) : r);
                uint32_t bit = 1u << (d + h);
                if (x < c->ta) { /* quadrant (0,0) */
                } else if (x < c->tab) { b |= bit; }
                else if (x < c->tabc) { a |= bit; }
                else { a |= bit; b |= bit; }
            }
        }
        if (c->scramble) { a = scramble_id(c, a); b = scramble_id(c, b); }
        c->u[e] = (int32_t)a; c->v[e] = (int32_t)b;
    }
}

gg_graph *gg_rmat(int scale, int edge_factor, double a, double b, double cq, uint64_t seed, int scramble,
                  int nthreads) {
    if (scale < 1 || scale > 30) return NULL;
    int64_t n = (int64_t)1 << scale;
    int64_t ne = n * (int64_t)edge_factor;
    rmat_ctx c;
    c.scale = scale; c.seed = seed; c.scramble = scramble;
    c.ta = (uint32_t)(a * 4294967296.0);
    c.tab = (uint32_t)((a + b) * 4294967296.0);
    c.tabc = (uint32_t)((a + b + cq) * 4294967296.0);
    for (int i = 0; i < 8; ++i) c.sm[i] = rng(seed, S_SCRAMBLE, (uint64_t)i);
    c.u = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
    c.v = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
    if (!c.u || !c.v) return NULL;
    parallel_for(ne, 1 << 16, nthreads, rmat_gen, &c);
    gg_graph *g = gg_from_edges(n, ne, c.u, c.v, 1, nthreads);
    free(c.u); free(c.v);
    return g;
}

/* ----------------------------------------------------------------- grid */
gg_graph *gg_grid(int rows, int cols, double delete_frac, double shortcut_frac, uint64_t seed,
                  int nthreads) {
    int64_t n = (int64_t)rows * cols;
    int64_t eh = (int64_t)rows * (cols - 1), ev = (int64_t)(rows - 1) * cols;
    int64_t e0 = eh + ev;
    int64_t nsc = (int64_t)floor(shortcut_frac * (double)e0 + 1e-9);
    uint64_t tdel = (delete_frac <= 0) ? 0 : (uint64_t)(delete_frac * 18446744073709551616.0);
    int32_t *u = (int32_t *)malloc((size_t)(e0 + nsc + 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(e0 + nsc + 1) * sizeof(int32_t));
    if (!u || !v) return NULL;
    int64_t k = 0;
    for (int64_t e = 0; e < e0; ++e) {
        if (tdel && rng(seed, S_GRID_DEL, (uint64_t)e) < tdel) continue;
        int64_t a, b;
        if (e < eh) { int64_t r = e / (cols - 1), c = e % (cols - 1); a = r * cols + c; b = a + 1; }
        else { int64_t f = e - eh; int64_t r = f / cols, c = f % cols; a = r * cols + c; b = a + cols; }
        u[k] = (int32_t)a; v[k] = (int32_t)b; ++k;
    }
    for (int64_t s = 0; s < nsc; ++s) {
        u[k] = (int32_t)bounded(rng(seed, S_GRID_SC, 2 * (uint64_t)s), (uint64_t)n);
        v[k] = (int32_t)bounded(rng(seed, S_GRID_SC, 2 * (uint64_t)s + 1), (uint64_t)n);
        ++k;
    }
    gg_graph *g = gg_from_edges(n, k, u, v, 1, nthreads);
    free(u); free(v);
    return g;
}

/* ------------------------------------------------------------------- BA */
/* Batagelj-Brandes: endpoint list M of length 2nm; the i-th new edge of
 * vertex v is (v, M[r]) with r uniform over the list written so far. */
static int64_t ba_edges(int64_t n, int m, uint64_t seed, uint64_t stream, int32_t *M) {
    int64_t len = 2 * n * (int64_t)m;
    for (int64_t v = 0; v < n; ++v) {
        for (int i = 0; i < m; ++i) {
            int64_t idx = 2 * (v * m + i);
            M[idx] = (int32_t)v;
            uint64_t r = bounded(rng(seed, stream, (uint64_t)idx), (uint64_t)idx + 1);
            M[idx + 1] = M[r];
        }
    }
    return len / 2;
}

gg_graph *gg_ba(int64_t n, int m, uint64_t seed, int nthreads) {
    int32_t *M = (int32_t *)malloc((size_t)(2 * n * (int64_t)m) * sizeof(int32_t));
    if (!M) return NULL;
    int64_t ne = ba_edges(n, m, seed, S_BA, M);
    /* split interleaved list into u/v */
    int32_t *u = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
    for (int64_t e = 0; e < ne; ++e) { u[e] = M[2 * e]; v[e] = M[2 * e + 1]; }
    free(M);
    gg_graph *g = gg_from_edges(n, ne, u, v, 1, nthreads);
    free(u); free(v);
    return g;
}

/* ------------------------------------------------------------------ RGG */
typedef struct {
    int64_t n; uint64_t seed; int64_t gsz; uint64_t r2; int64_t rint;
    uint32_t *x, *y; int64_t *cell_start; int32_t *cell_pts;
    int64_t *ecount; int32_t **eu, **ev; int64_t *ecap;
} rgg_ctx;

static void rgg_pairs(void *p, int64_t lo, int64_t hi, int tid) {
    rgg_ctx *c = (rgg_ctx *)p;
    for (int64_t cell = lo; cell < hi; ++cell) {
        int64_t cx = cell % c->gsz, cy = cell / c->gsz;
        for (int64_t i = c->cell_start[cell]; i < c->cell_start[cell + 1]; ++i) {
            int32_t a = c->cell_pts[i];
            for (int64_t dy = -1; dy <= 1; ++dy) for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t nx = cx + dx, ny = cy + dy;
                if (nx < 0 || ny < 0 || nx >= c->gsz || ny >= c->gsz) continue;
                int64_t nc = ny * c->gsz + nx;
                for (int64_t j = c->cell_start[nc]; j < c->cell_start[nc + 1]; ++j) {
                    int32_t b = c->cell_pts[j];
                    if (b <= a) continue;
                    int64_t ddx = (int64_t)c->x[a] - (int64_t)c->x[b];
                    int64_t ddy = (int64_t)c->y[a] - (int64_t)c->y[b];
                    uint64_t d2 = (uint64_t)(ddx * ddx) + (uint64_t)(ddy * ddy);
                    if (d2 <= c->r2) {
                        if (c->ecount[tid] == c->ecap[tid]) {
                            c->ecap[tid] = c->ecap[tid] * 2 + 1024;
                            c->eu[tid] = (int32_t *)realloc(c->eu[tid], (size_t)c->ecap[tid] * 4);
                            c->ev[tid] = (int32_t *)realloc(c->ev[tid], (size_t)c->ecap[tid] * 4);
                        }
                        c->eu[tid][c->ecount[tid]] = a; c->ev[tid][c->ecount[tid]] = b; c->ecount[tid]++;
                    }
                }
            }
        }
    }
}

gg_graph *gg_rgg(int64_t n, double avg_degree, uint64_t seed, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    const double L = 2147483648.0; /* lattice 2^31 */
    double r = sqrt(avg_degree / (3.14159265358979323846 * (double)n));
    rgg_ctx c;
    memset(&c, 0, sizeof c);
    c.n = n; c.seed = seed;
    c.rint = (int64_t)floor(r * L);
    c.r2 = (uint64_t)c.rint * (uint64_t)c.rint;
    c.gsz = (int64_t)floor(L / (double)(c.rint + 1));
    if (c.gsz < 1) c.gsz = 1;
    c.x = (uint32_t *)malloc((size_t)n * 4); c.y = (uint32_t *)malloc((size_t)n * 4);
    int64_t ncell = c.gsz * c.gsz;
    c.cell_start = (int64_t *)calloc((size_t)ncell + 1, 8);
    c.cell_pts = (int32_t *)malloc((size_t)n * 4);
    int64_t *cellof = (int64_t *)malloc((size_t)n * 8);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t h = rng(seed, S_RGG, (uint64_t)i);
        c.x[i] = (uint32_t)(h & 0x7FFFFFFFu);
        c.y[i] = (uint32_t)((h >> 32) & 0x7FFFFFFFu);
        int64_t gx = (int64_t)((uint64_t)c.x[i] * (uint64_t)c.gsz >> 31);
        int64_t gy = (int64_t)((uint64_t)c.y[i] * (uint64_t)c.gsz >> 31);
        cellof[i] = gy * c.gsz + gx;
        c.cell_start[cellof[i] + 1]++;
    }
    for (int64_t i = 0; i < ncell; ++i) c.cell_start[i + 1] += c.cell_start[i];
    int64_t *cur = (int64_t *)malloc((size_t)ncell * 8);
    memcpy(cur, c.cell_start, (size_t)ncell * 8);
    for (int64_t i = 0; i < n; ++i) c.cell_pts[cur[cellof[i]]++] = (int32_t)i;
    free(cur); free(cellof);
    c.ecount = (int64_t *)calloc(256, 8); c.ecap = (int64_t *)calloc(256, 8);
    c.eu = (int32_t **)calloc(256, sizeof(int32_t *)); c.ev = (int32_t **)calloc(256, sizeof(int32_t *));
    parallel_for(ncell, 256, nthreads, rgg_pairs, &c);
    int64_t ne = 0;
    for (int t = 0; t < nthreads; ++t) ne += c.ecount[t];
    int32_t *u = (int32_t *)malloc((size_t)(ne + 1) * 4), *v = (int32_t *)malloc((size_t)(ne + 1) * 4);
    int64_t k = 0;
    for (int t = 0; t < nthreads; ++t) {
        memcpy(u + k, c.eu[t], (size_t)c.ecount[t] * 4);
        memcpy(v + k, c.ev[t], (size_t)c.ecount[t] * 4);
        k += c.ecount[t];
        free(c.eu[t]); free(c.ev[t]);
    }
    gg_graph *g = gg_from_edges(n, ne, u, v, 1, nthreads);
    free(u); free(v); free(c.x); free(c.y); free(c.cell_start); free(c.cell_pts);
    free(c.ecount); free(c.ecap); free(c.eu); free(c.ev);
    return g;
}

/* ------------------------------------------------------ Erdos-Renyi G(n,M) */
gg_graph *gg_er(int64_t n, int64_t m, uint64_t seed, int directed, int nthreads) {
    int32_t *u = (int32_t *)malloc((size_t)(m + 1) * 4), *v = (int32_t *)malloc((size_t)(m + 1) * 4);
    for (int64_t e = 0; e < m; ++e) {
        u[e] = (int32_t)bounded(rng(seed, S_ER, 2 * (uint64_t)e), (uint64_t)n);
        v[e] = (int32_t)bounded(rng(seed, S_ER, 2 * (uint64_t)e + 1), (uint64_t)n);
    }
    gg_graph *g = gg_from_edges(n, m, u, v, directed ? 0 : 1, nthreads);
    free(u); free(v);
    return g;
}

/* -------------------------------------------------------------- sources */
/* k distinct vertices of nonzero out-degree drawn uniformly; returns the
 * number found (less than k only if fewer such vertices exist). */
int gg_sources(const int64_t *row_ptr, int64_t n, int k, uint64_t seed, int32_t *out) {
    int64_t nz = 0;
    for (int64_t v = 0; v < n; ++v) nz += (row_ptr[v + 1] > row_ptr[v]);
    if (nz < k) k = (int)nz;
    int found = 0;
    for (uint64_t i = 0; found < k; ++i) {
        int32_t v = (int32_t)bounded(rng(seed, S_SRC, i), (uint64_t)n);
        if (row_ptr[v + 1] == row_ptr[v]) continue;
        int dup = 0;
        for (int j = 0; j < found; ++j) if (out[j] == v) { dup = 1; break; }
        if (!dup) out[found++] = v;
    }
    return found;
}

/* ------------------------------------------ batch of small BA graphs */
typedef struct {
    int32_t g; int m; uint64_t seed; int64_t nmin, nmax;
    int64_t *sizes; gg_graph **graphs;
} batch_ctx;

static void batch_gen(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    batch_ctx *c = (batch_ctx *)p;
    for (int64_t i = lo; i < hi; ++i) {
        int64_t n = c->sizes[i];
        int32_t *M = (int32_t *)malloc((size_t)(2 * n * (int64_t)c->m) * sizeof(int32_t));
        int64_t ne = ba_edges(n, c->m, c->seed, (uint64_t)S_BATCH * 1000003ULL + (uint64_t)i, M);
        int32_t *u = (int32_t *)malloc((size_t)ne * 4), *v = (int32_t *)malloc((size_t)ne * 4);
        for (int64_t e = 0; e < ne; ++e) { u[e] = M[2 * e]; v[e] = M[2 * e + 1]; }
        free(M);
        c->graphs[i] = gg_from_edges(n, ne, u, v, 1, 1);
        free(u); free(v);
    }
}

/* g graphs, n drawn log-uniform in [nmin, nmax], attachment m. */
gg_batch *gg_ba_batch(int32_t g, int64_t nmin, int64_t nmax, int m, uint64_t seed, int nthreads) {
    batch_ctx c;
    c.g = g; c.m = m; c.seed = seed; c.nmin = nmin; c.nmax = nmax;
    c.sizes = (int64_t *)malloc((size_t)g * 8);
    c.graphs = (gg_graph **)calloc((size_t)g, sizeof(gg_graph *));
    double lmin = log((double)nmin), lmax = log((double)nmax);
    for (int32_t i = 0; i < g; ++i) {
        /* 53-bit uniform in [0,1) */
        double u01 = (double)(rng(seed, S_BATCH, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
        int64_t n = (int64_t)floor(exp(lmin + u01 * (lmax - lmin)));
        if (n < nmin) n = nmin;
        if (n > nmax) n = nmax;
        c.sizes[i] = n;
    }
    parallel_for(g, 4, nthreads, batch_gen, &c);
    gg_batch *b = (gg_batch *)calloc(1, sizeof(gg_batch));
    b->g = g;
    b->vtx_off = (int64_t *)malloc(((size_t)g + 1) * 8);
    b->edge_off = (int64_t *)malloc(((size_t)g + 1) * 8);
    int64_t tn = 0, te = 0;
    for (int32_t i = 0; i < g; ++i) {
        b->vtx_off[i] = tn; b->edge_off[i] = te;
        tn += c.graphs[i]->n; te += c.graphs[i]->nnz;
    }
    b->vtx_off[g] = tn; b->edge_off[g] = te;
    b->total_n = tn; b->total_nnz = te;
    b->row_ptr = (int64_t *)malloc(((size_t)tn + (size_t)g) * 8);
    b->col = (int32_t *)malloc((size_t)(te > 0 ? te : 1) * 4);
    for (int32_t i = 0; i < g; ++i) {
        gg_graph *gi = c.graphs[i];
        memcpy(b->row_ptr + b->vtx_off[i] + i, gi->row_ptr, ((size_t)gi->n + 1) * 8);
        memcpy(b->col + b->edge_off[i], gi->col, (size_t)gi->nnz * 4);
        gg_free(gi);
    }
    free(c.graphs); free(c.sizes);
    return b;
}
void gg_batch_free(gg_batch *b) {
    if (!b) return;
    free(b->vtx_off); free(b->edge_off); free(b->row_ptr); free(b->col); free(b);
}
int32_t gg_batch_g(const gg_batch *b) { return b->g; }
int64_t gg_batch_total_n(const gg_batch *b) { return b->total_n; }
int64_t gg_batch_total_nnz(const gg_batch *b) { return b->total_nnz; }
void gg_batch_copy(const gg_batch *b, int64_t *vtx_off, int64_t *edge_off, int64_t *row_ptr, int32_t *col) {
    memcpy(vtx_off, b->vtx_off, ((size_t)b->g + 1) * 8);
    memcpy(edge_off, b->edge_off, ((size_t)b->g + 1) * 8);
    memcpy(row_ptr, b->row_ptr, ((size_t)b->total_n + (size_t)b->g) * 8);
    memcpy(col, b->col, (size_t)b->total_nnz * 4);
}
