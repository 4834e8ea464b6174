// Vertex reordering on the device (§4).
//
// rcm: reverse Cuthill-McKee (§4.2).  Components are started, in order, from
//   the unvisited vertex of smallest (degree, id); each is visited level by
//   level.  In the serial algorithm a vertex joins the order when its first
//   already-ordered neighbour is dequeued, and the children of one vertex are
//   appended by ascending (degree, id); so the vertices of a new level are
//   exactly the order sorted by (position of the earliest-positioned
//   neighbour in the previous level, degree, id).  Each level is therefore:
//   expand (atomicMin of the parent position), two stable radix sorts, and a
//   position assignment -- the serial order, reproduced exactly.  Degree-0
//   vertices are singleton components and come first (smallest degree).
//
// jaccard: JaccardWithWindows (§4.1, Algorithm 1).  One CTA per window; the
//   greedy steps of a window are sequential, the work inside a step (rows of
//   the chosen column, their columns inside the window, the argmax over the
//   candidate list Q) is spread over the CTA.  Tie-breaks: lowest column
//   index; the ratio inter / (|R| + deg - inter) is compared as exact 64-bit
//   cross-products.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "prim.cuh"
#include "reorder.h"

namespace {

constexpr int TB = 256;

unsigned gridn(int64_t items, int per = TB, int cap = 1 << 16) {
    int64_t b = (items + per - 1) / per;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

struct Tmp {
    cudaStream_t st;
    std::vector<void *> ptrs;
    bool bad = false;
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, count * sizeof(T) + 16, st) != cudaSuccess) { bad = true; return nullptr; }
        ptrs.push_back(p);
        return (T *)p;
    }
    ~Tmp() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

// ------------------------------------------------------------- clean CSR
__global__ void k_arc_keys(const long long *__restrict__ rp, const int *__restrict__ col, int64_t n, int B,
                           unsigned long long *keys) {
    const int lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw)
        for (long long p = rp[j] + lane; p < rp[j + 1]; p += 32) {
            const int i = col[p];
            keys[p] = ((int64_t)i == j) ? ~0ull : (((unsigned long long)j << B) | (unsigned long long)i);
        }
}

// both orientations of every arc (a directed graph's symmetrised pattern,
// G + G^T, on which the orderings run): keys 2p and 2p + 1
__global__ void k_arc_keys_sym(const long long *__restrict__ rp, const int *__restrict__ col, int64_t n, int B,
                               unsigned long long *keys) {
    const int lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw)
        for (long long p = rp[j] + lane; p < rp[j + 1]; p += 32) {
            const int i = col[p];
            const bool loop = (int64_t)i == j;
            keys[2 * p] = loop ? ~0ull : (((unsigned long long)j << B) | (unsigned long long)i);
            keys[2 * p + 1] = loop ? ~0ull : (((unsigned long long)i << B) | (unsigned long long)j);
        }
}

// in-degrees of a duplicate-free CSR
__global__ void k_in_degree(const int *__restrict__ col, int64_t m, int *indeg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += stride) atomicAdd(&indeg[col[p]], 1);
}

__global__ void k_uniq_flags(const unsigned long long *__restrict__ k, int64_t m, int *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += stride)
        flag[p] = (k[p] != ~0ull && (p == 0 || k[p] != k[p - 1])) ? 1 : 0;
}

__global__ void k_uniq_scatter(const unsigned long long *__restrict__ k, const int *__restrict__ flag,
                               const long long *__restrict__ pos, int64_t m, int B, int *col, int *deg) {
    const unsigned long long mask = (1ull << B) - 1ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += stride)
        if (flag[p]) {
            col[pos[p]] = (int)(k[p] & mask);
            atomicAdd(&deg[k[p] >> B], 1);
        }
}

__global__ void k_deg_to_ll(const int *__restrict__ deg, int64_t n, long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = deg[v];
}

// ------------------------------------------------------------------- RCM
__global__ void k_deg_keys(const int *__restrict__ deg, int64_t n, unsigned long long *keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        keys[v] = ((unsigned long long)deg[v] << 32) | (unsigned long long)v;
}

__global__ void k_init_rcm(int64_t n, int *pos, int *parent, int *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        pos[v] = -1;
        parent[v] = 0x7FFFFFFF;
        flag[v] = 0;
    }
}

// the first z entries of the (degree, id)-sorted list have degree 0
__global__ void k_place_isolated(const unsigned long long *__restrict__ sorted, int64_t z, int *pos, int *order) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < z; k += stride) {
        const int v = (int)(sorted[k] & 0xFFFFFFFFull);
        pos[v] = (int)k;
        order[k] = v;
    }
}

__global__ void k_count_deg0(const int *__restrict__ deg, int64_t n, unsigned long long *z) {
    unsigned long long c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) c += deg[v] == 0;
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(z, c);
}

// smallest k in [from, to) whose vertex has no position yet
__global__ void k_first_unplaced(const unsigned long long *__restrict__ sorted, const int *__restrict__ pos,
                                 int64_t from, int64_t to, unsigned long long *best) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < to; k += stride) {
        const int v = (int)(sorted[k] & 0xFFFFFFFFull);
        if (pos[v] < 0) atomicMin(best, (unsigned long long)k);
    }
}

__global__ void k_start(const unsigned long long *__restrict__ sorted, long long k, int p, int *pos, int *order) {
    const int v = (int)(sorted[k] & 0xFFFFFFFFull);
    pos[v] = p;
    order[p] = v;
}

// vertices at positions [f0, f1) expand; unplaced neighbours record the
// smallest parent position and join the candidate list once
__global__ void k_expand_level(const long long *__restrict__ rp, const int *__restrict__ col,
                               const int *__restrict__ order, int f0, int f1, const int *__restrict__ pos,
                               int *parent, int *flag, int *cand, int *ncand) {
    const int lane = lane_id();
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int p = f0 + gw; p < f1; p += nw) {
        const int v = order[p];
        for (long long e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const int w = col[e];
            if (pos[w] >= 0) continue;
            atomicMin(&parent[w], p);
            if (atomicCAS(&flag[w], 0, 1) == 0) cand[atomicAdd(ncand, 1)] = w;
        }
    }
}

__global__ void k_cand_keys(const int *__restrict__ cand, int c, const int *__restrict__ deg,
                            unsigned long long *keys) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
        const int w = cand[k];
        keys[k] = ((unsigned long long)deg[w] << 32) | (unsigned long long)(unsigned)w;
    }
}
__global__ void k_parent_keys(const unsigned long long *__restrict__ sorted, int c, const int *__restrict__ parent,
                              unsigned long long *pkeys, unsigned *vals) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
        const int w = (int)(sorted[k] & 0xFFFFFFFFull);
        pkeys[k] = (unsigned long long)parent[w];
        vals[k] = (unsigned)w;
    }
}
__global__ void k_assign(const unsigned *__restrict__ vals, int c, int base, int *pos, int *order) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
        const int w = (int)vals[k];
        pos[w] = base + k;
        order[base + k] = w;
    }
}

// small levels: one CTA sorts (parent, degree, id) triples with a bitonic network
constexpr int SMALL_SORT = 2048;
__global__ void __launch_bounds__(1024) k_small_level_sort(const int *__restrict__ cand, int c,
                                                           const int *__restrict__ parent, const int *__restrict__ deg,
                                                           int base, int *pos, int *order) {
    __shared__ unsigned long long k1[SMALL_SORT];   // parent << 32 | degree
    __shared__ int k2[SMALL_SORT];                  // id
    int P2 = 1;
    while (P2 < c) P2 <<= 1;
    for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        if (i < c) {
            const int w = cand[i];
            k1[i] = ((unsigned long long)(unsigned)parent[w] << 32) | (unsigned)deg[w];
            k2[i] = w;
        } else {
            k1[i] = ~0ull;
            k2[i] = 0x7FFFFFFF;
        }
    }
    __syncthreads();
    for (int size = 2; size <= P2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const bool gt = k1[i] > k1[j] || (k1[i] == k1[j] && k2[i] > k2[j]);
                    if (gt == up) {
                        const unsigned long long t1 = k1[i]; k1[i] = k1[j]; k1[j] = t1;
                        const int t2 = k2[i]; k2[i] = k2[j]; k2[j] = t2;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        pos[k2[i]] = base + i;
        order[base + i] = k2[i];
    }
}

__global__ void k_reverse(const int *__restrict__ pos, int64_t n, int *new_of_old) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        new_of_old[v] = (int)(n - 1 - pos[v]);
}

// --------------------------------------------------------------- Jaccard
struct JacParams {
    const long long *rp;
    const int *col;       // sorted rows
    const int *deg;
    const unsigned long long *by_degree;  // per window: (window << 32 | ~deg) sorted; low id recovered below
    const int *by_degree_id;
    int64_t n;
    int W;
    int sigma;            // columns per slice set
    int nwin;
    int *inter;           // per block: W
    int *qlist;           // per block: W
    unsigned *rbits;      // per block: ceil(n/32) words
    int *new_of_old;
};

// first index in the sorted row i with col >= lo
__device__ __forceinline__ long long lower_bound_row(const int *col, long long a, long long b, int lo) {
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (col[m] < lo) a = m + 1;
        else b = m;
    }
    return a;
}

__global__ void __launch_bounds__(1024, 1) k_jaccard(JacParams P) {
    extern __shared__ unsigned s_assigned[];          // W bits
    __shared__ int s_j, s_qcount, s_rsize, s_ptr, s_chosen[32];
    __shared__ unsigned long long s_bnum[32], s_bden[32];
    __shared__ int s_bj[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int W = P.W;
    int *inter = P.inter + (size_t)blockIdx.x * W;
    int *qlist = P.qlist + (size_t)blockIdx.x * W;
    unsigned *rbits = P.rbits + (size_t)blockIdx.x * ((P.n + 31) / 32);

    for (int w = blockIdx.x; w < P.nwin; w += gridDim.x) {
        const int64_t ws = (int64_t)w * W;
        const int64_t we = (ws + W < P.n) ? ws + W : P.n;
        const int wn = (int)(we - ws);
        for (int i = tid; i < (W + 31) / 32; i += nthr) s_assigned[i] = 0u;
        for (int i = tid; i < W; i += nthr) inter[i] = 0;
        if (tid == 0) { s_qcount = 0; s_ptr = 0; }
        __syncthreads();
        const int nss = (wn + P.sigma - 1) / P.sigma;
        for (int s = 0; s < nss; ++s) {
            const int64_t ss = ws + (int64_t)s * P.sigma;
            const int64_t se = (ss + P.sigma < we) ? ss + P.sigma : we;
            int nch = 0;
            for (int64_t slot = ss; slot < se; ++slot) {
                // ---- choose the column for this slot
                const bool seed = slot == ss;
                int qvalid = 0;
                if (!seed) {
                    // argmax over Q of inter / (|R| + deg - inter), lowest index on ties
                    unsigned long long bnum = 0, bden = 1;
                    int bj = 0x7FFFFFFF;
                    const int qc = s_qcount;
                    const unsigned long long R = (unsigned long long)s_rsize;
                    for (int k = tid; k < qc; k += nthr) {
                        const int jj = qlist[k];
                        const int lj = (int)(jj - ws);
                        if (s_assigned[lj >> 5] >> (lj & 31) & 1u) continue;
                        const unsigned long long num = (unsigned long long)inter[lj];
                        const unsigned long long den = R + (unsigned long long)P.deg[jj] - num;
                        const bool better = (bj == 0x7FFFFFFF) || num * bden > bnum * den ||
                                            (num * bden == bnum * den && jj < bj);
                        if (better) { bnum = num; bden = den; bj = jj; }
                    }
                    // warp then block reduction with the same order
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long on = __shfl_xor_sync(FULL_MASK, bnum, o);
                        const unsigned long long od = __shfl_xor_sync(FULL_MASK, bden, o);
                        const int oj = __shfl_xor_sync(FULL_MASK, bj, o);
                        const bool take = oj != 0x7FFFFFFF &&
                                          (bj == 0x7FFFFFFF || on * bden > bnum * od || (on * bden == bnum * od && oj < bj));
                        if (take) { bnum = on; bden = od; bj = oj; }
                    }
                    if ((tid & 31) == 0) { s_bnum[tid >> 5] = bnum; s_bden[tid >> 5] = bden; s_bj[tid >> 5] = bj; }
                    __syncthreads();
                    if (tid == 0) {
                        int best = 0x7FFFFFFF;
                        unsigned long long cn = 0, cd = 1;
                        for (int k = 0; k < nthr / 32; ++k) {
                            const int oj = s_bj[k];
                            if (oj == 0x7FFFFFFF) continue;
                            const unsigned long long on = s_bnum[k], od = s_bden[k];
                            if (best == 0x7FFFFFFF || on * cd > cn * od || (on * cd == cn * od && oj < best)) {
                                best = oj; cn = on; cd = od;
                            }
                        }
                        s_j = best;
                    }
                    __syncthreads();
                    qvalid = s_j != 0x7FFFFFFF;
                }
                if (tid == 0) {
                    int j = s_j;
                    if (seed || !qvalid) {
                        // highest-degree unassigned column of the window
                        int p = s_ptr;
                        for (;;) {
                            const int cj = P.by_degree_id[ws + p];
                            const int lj = (int)(cj - ws);
                            if (!(s_assigned[lj >> 5] >> (lj & 31) & 1u)) { j = cj; break; }
                            ++p;
                        }
                        s_ptr = p;
                    }
                    const int lj = (int)(j - ws);
                    s_assigned[lj >> 5] |= 1u << (lj & 31);
                    P.new_of_old[j] = (int)slot;
                    s_j = j;
                    s_chosen[nch] = j;
                    if (seed) s_rsize = 0;
                }
                __syncthreads();
                const int j = s_j;
                ++nch;
                // ---- R gains the new rows of j; their columns in the window gain inter
                for (long long e = P.rp[j] + tid; e < P.rp[j + 1]; e += nthr) {
                    const int i = P.col[e];
                    const unsigned old = atomicOr(&rbits[i >> 5], 1u << (i & 31));
                    if (old >> (i & 31) & 1u) continue;
                    atomicAdd(&s_rsize, 1);
                    const long long a = lower_bound_row(P.col, P.rp[i], P.rp[i + 1], (int)ws);
                    for (long long f = a; f < P.rp[i + 1]; ++f) {
                        const int jj = P.col[f];
                        if (jj >= we) break;
                        const int lj = (int)(jj - ws);
                        if (s_assigned[lj >> 5] >> (lj & 31) & 1u) continue;
                        if (atomicAdd(&inter[lj], 1) == 0) qlist[atomicAdd(&s_qcount, 1)] = jj;
                    }
                }
                __syncthreads();
            }
            // ---- reset inter, Q and R for the next slice set
            const int qc = s_qcount;
            for (int k = tid; k < qc; k += nthr) inter[qlist[k] - ws] = 0;
            for (int c = 0; c < nch; ++c) {
                const int jc = s_chosen[c];
                for (long long e = P.rp[jc] + tid; e < P.rp[jc + 1]; e += nthr) {
                    const int i = P.col[e];
                    rbits[i >> 5] = 0u;
                }
            }
            __syncthreads();
            if (tid == 0) s_qcount = 0;
            __syncthreads();
        }
    }
}

__global__ void k_window_keys(const int *__restrict__ deg, int64_t n, int W, unsigned long long *keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long w = (unsigned long long)(v / W);
        keys[v] = (w << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)deg[v]);
    }
}

}  // namespace

// Clean CSR of the input (rows sorted, duplicates and self loops removed).
// The duplicate- and loop-free CSR of (rp, col), rows sorted; sym: of its
// symmetrised pattern (every arc in both directions).
static blest_status clean_csr(cudaStream_t st, Tmp &T, const long long *rp, const int *col, int64_t n,
                              int64_t nnz_in, long long **rp_out, int **col_out, int **deg_out, bool sym = false) {
    const int B = ceil_log2_i64(n) > 0 ? ceil_log2_i64(n) : 1;
    const int64_t nnz = sym ? 2 * nnz_in : nnz_in;
    unsigned long long *k = T.get<unsigned long long>((size_t)nnz + 1);
    unsigned long long *ka = T.get<unsigned long long>((size_t)nnz + 1);
    long long *hist = T.get<long long>(radix_hist_elems(nnz));
    long long *stmp = T.get<long long>(scan_tmp_elems(nnz > n ? nnz : n) + scan_tmp_elems((int64_t)radix_hist_elems(nnz)) + 32);
    int *flag = T.get<int>((size_t)nnz + 1);
    long long *pos = T.get<long long>((size_t)nnz + 2);
    int *c2 = T.get<int>((size_t)nnz + 1);
    int *deg = T.get<int>((size_t)n + 1);
    long long *deg64 = T.get<long long>((size_t)n + 2);
    long long *rp2 = T.get<long long>((size_t)n + 2);
    if (T.bad) return BLEST_ERR_OOM;
    cudaMemsetAsync(deg, 0, ((size_t)n + 1) * 4, st);
    if (sym) k_arc_keys_sym<<<gridn(n * 32), TB, 0, st>>>(rp, col, n, B, k);
    else k_arc_keys<<<gridn(n * 32), TB, 0, st>>>(rp, col, n, B, k);
    if (radix_sort_u64(k, nullptr, ka, nullptr, nnz, 2 * B + 1, hist, stmp, st) != cudaSuccess) return BLEST_ERR_CUDA;
    k_uniq_flags<<<gridn(nnz), TB, 0, st>>>(k, nnz, flag);
    if (scan_exclusive_i32_to_i64(flag, pos, nnz, stmp, st) != cudaSuccess) return BLEST_ERR_CUDA;
    k_uniq_scatter<<<gridn(nnz), TB, 0, st>>>(k, flag, pos, nnz, B, c2, deg);
    k_deg_to_ll<<<gridn(n), TB, 0, st>>>(deg, n, deg64);
    if (scan_exclusive_i64(deg64, rp2, n, stmp, st) != cudaSuccess) return BLEST_ERR_CUDA;
    *rp_out = rp2;
    *col_out = c2;
    *deg_out = deg;
    return cudaGetLastError() == cudaSuccess ? BLEST_OK : BLEST_ERR_CUDA;
}

static blest_status rcm_order(blest_graph *h, Tmp &T, const long long *rp, const int *col, const int *deg,
                              int64_t n, int *new_of_old) {
    cudaStream_t st = h->stream;
    int maxdeg_bits = 32;
    unsigned long long *keys = T.get<unsigned long long>((size_t)n + 1);
    unsigned long long *kalt = T.get<unsigned long long>((size_t)n + 1);
    unsigned long long *pk = T.get<unsigned long long>((size_t)n + 1);
    unsigned *pv = T.get<unsigned>((size_t)n + 1);
    unsigned *pva = T.get<unsigned>((size_t)n + 1);
    long long *hist = T.get<long long>(radix_hist_elems(n));
    long long *stmp = T.get<long long>(scan_tmp_elems((int64_t)radix_hist_elems(n)) + 32);
    int *pos = T.get<int>((size_t)n + 1);
    int *parent = T.get<int>((size_t)n + 1);
    int *flag = T.get<int>((size_t)n + 1);
    int *order = T.get<int>((size_t)n + 1);
    int *cand = T.get<int>((size_t)n + 1);
    int *ncand = T.get<int>(1);
    unsigned long long *scal = T.get<unsigned long long>(2);
    unsigned long long *sorted_deg = T.get<unsigned long long>((size_t)n + 1);
    if (T.bad) return BLEST_ERR_OOM;
    const int B = ceil_log2_i64(n) > 0 ? ceil_log2_i64(n) : 1;
    k_deg_keys<<<gridn(n), TB, 0, st>>>(deg, n, sorted_deg);
    if (radix_sort_u64(sorted_deg, nullptr, kalt, nullptr, n, 32 + maxdeg_bits, hist, stmp, st) != cudaSuccess)
        return BLEST_ERR_CUDA;
    k_init_rcm<<<gridn(n), TB, 0, st>>>(n, pos, parent, flag);
    cudaMemsetAsync(scal, 0, 16, st);
    k_count_deg0<<<gridn(n, TB, 4096), TB, 0, st>>>(deg, n, scal);
    unsigned long long z = 0;
    cudaMemcpyAsync(&z, scal, 8, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
    if (z) k_place_isolated<<<gridn((int64_t)z), TB, 0, st>>>(sorted_deg, (int64_t)z, pos, order);
    int64_t next = (int64_t)z, ptr = (int64_t)z;
    const int64_t WIN = 1 << 16;
    while (next < n) {
        // next start: the first unplaced vertex of the (degree, id) order
        unsigned long long best = ~0ull;
        while (best == ~0ull && ptr < n) {
            const int64_t to = ptr + WIN < n ? ptr + WIN : n;
            cudaMemcpyAsync(scal, &best, 8, cudaMemcpyHostToDevice, st);
            k_first_unplaced<<<gridn(to - ptr), TB, 0, st>>>(sorted_deg, pos, ptr, to, scal);
            cudaMemcpyAsync(&best, scal, 8, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
            if (best == ~0ull) ptr = to;
        }
        if (best == ~0ull) return BLEST_ERR_INTERNAL;
        ptr = (int64_t)best;
        k_start<<<1, 1, 0, st>>>(sorted_deg, (long long)best, (int)next, pos, order);
        int64_t f0 = next, f1 = next + 1;
        next += 1;
        while (f1 > f0) {
            cudaMemsetAsync(ncand, 0, 4, st);
            k_expand_level<<<gridn((f1 - f0) * 32, TB, 8192), TB, 0, st>>>(rp, col, order, (int)f0, (int)f1, pos,
                                                                             parent, flag, cand, ncand);
            int c = 0;
            cudaMemcpyAsync(&c, ncand, 4, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
            if (c == 0) break;
            if (c <= SMALL_SORT) {
                k_small_level_sort<<<1, 1024, 0, st>>>(cand, c, parent, deg, (int)next, pos, order);
            } else {
                k_cand_keys<<<gridn(c), TB, 0, st>>>(cand, c, deg, keys);
                if (radix_sort_u64(keys, nullptr, kalt, nullptr, c, 32 + maxdeg_bits, hist, stmp, st) != cudaSuccess)
                    return BLEST_ERR_CUDA;
                k_parent_keys<<<gridn(c), TB, 0, st>>>(keys, c, parent, pk, pv);
                if (radix_sort_u64(pk, pv, kalt, pva, c, B + 1, hist, stmp, st) != cudaSuccess) return BLEST_ERR_CUDA;
                k_assign<<<gridn(c), TB, 0, st>>>(pv, c, (int)next, pos, order);
            }
            f0 = next;
            f1 = next + c;
            next += c;
        }
    }
    k_reverse<<<gridn(n), TB, 0, st>>>(pos, n, new_of_old);
    return cudaGetLastError() == cudaSuccess ? BLEST_OK : BLEST_ERR_CUDA;
}

static blest_status jaccard_order(blest_graph *h, Tmp &T, const long long *rp, const int *col, const int *deg,
                                  int64_t n, int W, int *new_of_old) {
    cudaStream_t st = h->stream;
    const int nwin = (int)((n + W - 1) / W);
    unsigned long long *keys = T.get<unsigned long long>((size_t)n + 1);
    unsigned long long *kalt = T.get<unsigned long long>((size_t)n + 1);
    unsigned *ids = T.get<unsigned>((size_t)n + 1);
    unsigned *idsa = T.get<unsigned>((size_t)n + 1);
    long long *hist = T.get<long long>(radix_hist_elems(n));
    long long *stmp = T.get<long long>(scan_tmp_elems((int64_t)radix_hist_elems(n)) + 32);
    if (T.bad) return BLEST_ERR_OOM;
    // per window: columns by decreasing degree, lowest id first on ties (stable sort of id order)
    k_window_keys<<<gridn(n), TB, 0, st>>>(deg, n, W, keys);
    {
        std::vector<unsigned> idh((size_t)n);
        for (int64_t v = 0; v < n; ++v) idh[(size_t)v] = (unsigned)v;
        cudaMemcpyAsync(ids, idh.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st);
        const int wb = ceil_log2_i64(nwin) > 0 ? ceil_log2_i64(nwin) : 1;
        if (radix_sort_u64(keys, ids, kalt, idsa, n, 32 + wb, hist, stmp, st) != cudaSuccess) return BLEST_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(1, std::min(nwin, sms));
    const int64_t words = (n + 31) / 32;
    int *inter = T.get<int>((size_t)blocks * W);
    int *qlist = T.get<int>((size_t)blocks * W);
    unsigned *rbits = T.get<unsigned>((size_t)blocks * words);
    if (T.bad) return BLEST_ERR_OOM;
    cudaMemsetAsync(rbits, 0, (size_t)blocks * words * 4, st);
    JacParams P;
    P.rp = rp;
    P.col = col;
    P.deg = deg;
    P.by_degree = keys;
    P.by_degree_id = (const int *)ids;
    P.n = n;
    P.W = W;
    P.sigma = h->sigma;
    P.nwin = nwin;
    P.inter = inter;
    P.qlist = qlist;
    P.rbits = rbits;
    P.new_of_old = new_of_old;
    const size_t smem = (size_t)((W + 31) / 32) * 4;
    if (smem > 200 * 1024) return BLEST_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(k_jaccard, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jaccard<<<blocks, 1024, smem, st>>>(P);
    if (cudaGetLastError() != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
    return BLEST_OK;
}

// ------------------------------------------------ scale-free-like test
// The §4.2 footnote: a degree distribution is heavy-tailed when (a) the top
// 1 % of vertices hold >= 5 % and the top 10 % >= 40 % of the total degree,
// or (b) a least-squares line through the log-log degree histogram over
// k >= 5 has slope -gamma with R^2 >= 0.70 and gamma in [1, 5].  The
// histogram is built on the device; both tests read only the histogram
// (the top-p % sums walk it from the highest degree down), so the host part
// is O(max degree).  Top p % = floor(p n / 100) vertices, at least one; the
// fit takes every k >= 5 with h(k) > 0, unweighted, and needs two points.

__global__ void k_neg_check(const int *__restrict__ deg, int64_t n, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (deg[v] < 0) atomicExch(bad, 1);
}

__global__ void k_deg_max(const int *__restrict__ deg, int64_t n, int *mx) {
    int m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) m = max(m, deg[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL_MASK, m, o));
    if (lane_id() == 0 && m) atomicMax(mx, m);
}

// hist[k] = #vertices of degree k; degrees below SMALL_BINS count in shared
// memory first (most vertices of a skewed graph have small degrees, so
// global atomics on those bins would serialise)
constexpr int SMALL_BINS = 2048;
__global__ void k_deg_hist(const int *__restrict__ deg, int64_t n, unsigned long long *hist) {
    __shared__ unsigned sh[SMALL_BINS];
    for (int i = threadIdx.x; i < SMALL_BINS; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int d = deg[v];
        if (d < SMALL_BINS) atomicAdd(&sh[d], 1u);
        else atomicAdd(&hist[d], 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SMALL_BINS; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

static void report_from_hist(const std::vector<unsigned long long> &h, int64_t n, blest_degree_report *r) {
    memset(r, 0, sizeof *r);
    long long tot = 0;
    for (size_t k = 0; k < h.size(); ++k) tot += (long long)k * (long long)h[k];
    const long long n1 = std::max<long long>(1, n / 100), n10 = std::max<long long>(1, n / 10);
    if (n > 0 && tot > 0) {
        long long take1 = n1, take10 = n10, s1 = 0, s10 = 0;
        for (size_t kk = h.size(); kk-- > 0;) {
            const long long c = (long long)h[kk];
            const long long a = std::min(c, take1), b = std::min(c, take10);
            s1 += a * (long long)kk;
            s10 += b * (long long)kk;
            take1 -= a;
            take10 -= b;
            if (take10 == 0) break;
        }
        r->top1 = (double)s1 / (double)tot;
        r->top10 = (double)s10 / (double)tot;
    }
    r->concentrated = (r->top1 >= 0.05 && r->top10 >= 0.40) ? 1 : 0;
    // least squares of y = ln h(k) on x = ln k over k >= 5, h(k) > 0
    std::vector<double> xs, ys;
    for (size_t k = 5; k < h.size(); ++k)
        if (h[k]) {
            xs.push_back(std::log((double)k));
            ys.push_back(std::log((double)h[k]));
        }
    r->points = (int32_t)xs.size();
    r->gamma = NAN;
    r->r2 = NAN;
    if (xs.size() >= 2) {
        double mx = 0, my = 0;
        for (size_t i = 0; i < xs.size(); ++i) { mx += xs[i]; my += ys[i]; }
        mx /= (double)xs.size();
        my /= (double)xs.size();
        double sxx = 0, sxy = 0, syy = 0;
        for (size_t i = 0; i < xs.size(); ++i) {
            sxx += (xs[i] - mx) * (xs[i] - mx);
            sxy += (xs[i] - mx) * (ys[i] - my);
            syy += (ys[i] - my) * (ys[i] - my);
        }
        if (sxx > 0) {
            const double slope = sxy / sxx, icpt = my - slope * mx;
            double ssr = 0;
            for (size_t i = 0; i < xs.size(); ++i) {
                const double e = ys[i] - (slope * xs[i] + icpt);
                ssr += e * e;
            }
            r->gamma = -slope;
            r->r2 = syy > 0 ? 1.0 - ssr / syy : NAN;
        }
    }
    r->powerlaw = (std::isfinite(r->gamma) && std::isfinite(r->r2) && r->r2 >= 0.70 && r->gamma >= 1.0 &&
                   r->gamma <= 5.0) ? 1 : 0;
    r->heavy = (r->concentrated || r->powerlaw) ? 1 : 0;
}

// The report of one device degree array (n entries).
static blest_status degree_report(cudaStream_t st, Tmp &T, const int *deg, int64_t n, blest_degree_report *r) {
    int *mx = T.get<int>(1);
    if (T.bad) return BLEST_ERR_OOM;
    cudaMemsetAsync(mx, 0, 4, st);
    k_deg_max<<<gridn(n, TB, 4096), TB, 0, st>>>(deg, n, mx);
    int maxdeg = 0;
    cudaMemcpyAsync(&maxdeg, mx, 4, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
    const size_t bins = (size_t)std::max(maxdeg + 1, SMALL_BINS);
    unsigned long long *hist = T.get<unsigned long long>(bins);
    if (T.bad) return BLEST_ERR_OOM;
    cudaMemsetAsync(hist, 0, bins * 8, st);
    k_deg_hist<<<gridn(n, TB, 4096), TB, 0, st>>>(deg, n, hist);
    std::vector<unsigned long long> hh((size_t)maxdeg + 1);
    cudaMemcpyAsync(hh.data(), hist, hh.size() * 8, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return BLEST_ERR_CUDA;
    report_from_hist(hh, n, r);
    return BLEST_OK;
}

// out_deg / in_deg: device arrays (in_deg may be null: undirected)
static blest_status scale_free_report(cudaStream_t st, Tmp &T, const int *out_deg, const int *in_deg, int64_t n,
                                      blest_scale_free_report *rep) {
    memset(rep, 0, sizeof *rep);
    blest_status s = degree_report(st, T, out_deg, n, &rep->out_deg);
    if (s != BLEST_OK) return s;
    if (in_deg) {
        if ((s = degree_report(st, T, in_deg, n, &rep->in_deg)) != BLEST_OK) return s;
    } else {
        rep->in_deg = rep->out_deg;
    }
    rep->scale_free = (rep->out_deg.heavy || rep->in_deg.heavy) ? 1 : 0;
    return BLEST_OK;
}

blest_status reorder_graph(blest_graph *h, const long long *rp, const int *col, int64_t n, int64_t nnz,
                           const blest_build_opts *o, int *new_of_old, int *applied) {
    Tmp T{h->stream};
    long long *rp2 = nullptr;
    int *col2 = nullptr, *deg = nullptr;
    blest_status st = clean_csr(h->stream, T, rp, col, n, nnz, &rp2, &col2, &deg);
    if (st != BLEST_OK) return st;
    int which = o->reorder;
    if (which == BLEST_REORDER_AUTO) {
        int *indeg = nullptr;
        if (h->directed) {
            long long m = 0;
            cudaMemcpyAsync(&m, rp2 + n, 8, cudaMemcpyDeviceToHost, h->stream);
            indeg = T.get<int>((size_t)n + 1);
            if (T.bad) return BLEST_ERR_OOM;
            cudaMemsetAsync(indeg, 0, (size_t)n * 4, h->stream);
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
            if (m > 0) k_in_degree<<<gridn(m), TB, 0, h->stream>>>(col2, m, indeg);
        }
        blest_scale_free_report rep;
        if ((st = scale_free_report(h->stream, T, deg, indeg, n, &rep)) != BLEST_OK) return st;
        which = rep.scale_free ? BLEST_REORDER_JACCARD : BLEST_REORDER_RCM;
    }
    if (h->directed) {
        // the orderings run on the symmetrised pattern G + G^T (RCM is defined
        // for symmetric patterns; the permutation changes speed, never levels)
        if ((st = clean_csr(h->stream, T, rp, col, n, nnz, &rp2, &col2, &deg, true)) != BLEST_OK) return st;
    }
    if (which == BLEST_REORDER_RCM) st = rcm_order(h, T, rp2, col2, deg, n, new_of_old);
    else if (which == BLEST_REORDER_JACCARD) st = jaccard_order(h, T, rp2, col2, deg, n, o->jaccard_window, new_of_old);
    else return BLEST_ERR_INVALID;
    if (st != BLEST_OK) return st;
    *applied = which;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? BLEST_OK : BLEST_ERR_CUDA;
}

// ---- C ABI: the classifier on caller degree arrays (host or device)
extern "C" blest_status blest_scale_free_test(const int32_t *out_deg, const int32_t *in_deg, int64_t n,
                                              blest_scale_free_report *out) {
    if (!out_deg || !out || n < 1 || n >= (1ll << 31)) return BLEST_ERR_INVALID;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return BLEST_ERR_CUDA;
    blest_status s = BLEST_OK;
    {
        Tmp T{st};
        int *d_out = T.get<int>((size_t)n), *d_in = in_deg ? T.get<int>((size_t)n) : nullptr;
        if (T.bad) s = BLEST_ERR_OOM;
        if (s == BLEST_OK && cudaMemcpyAsync(d_out, out_deg, (size_t)n * 4, cudaMemcpyDefault, st) != cudaSuccess)
            s = BLEST_ERR_CUDA;
        if (s == BLEST_OK && in_deg &&
            cudaMemcpyAsync(d_in, in_deg, (size_t)n * 4, cudaMemcpyDefault, st) != cudaSuccess)
            s = BLEST_ERR_CUDA;
        int *d_bad = s == BLEST_OK ? T.get<int>(1) : nullptr;
        if (s == BLEST_OK && T.bad) s = BLEST_ERR_OOM;
        if (s == BLEST_OK) {   // degrees must be non-negative
            cudaMemsetAsync(d_bad, 0, 4, st);
            k_neg_check<<<gridn(n, TB, 4096), TB, 0, st>>>(d_out, n, d_bad);
            if (d_in) k_neg_check<<<gridn(n, TB, 4096), TB, 0, st>>>(d_in, n, d_bad);
            int bad = 0;
            cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) s = BLEST_ERR_CUDA;
            else if (bad) s = BLEST_ERR_INVALID;
        }
        if (s == BLEST_OK) s = scale_free_report(st, T, d_out, d_in, n, out);
        cudaStreamSynchronize(st);
    }
    cudaStreamDestroy(st);
    return s;
}
