// Graph build on the device: CSR validation, optional reordering, BVSS
// packing (§3.1), update divergence (§4.2) and the in-neighbour CSR used by
// bottom-up levels (Algorithm 4).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "handle.h"
#include "prim.cuh"
#include "reorder.h"

namespace {

constexpr int TB = 256;

static inline unsigned grid_for(int64_t items, int per_block = TB, int cap = 1 << 20) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// ---- validation: row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz, cols in range
__global__ void k_validate(const long long *__restrict__ rp, const int *__restrict__ col, int64_t n,
                           int64_t nnz, int *bad) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = tid; v < n; v += stride)
        if (rp[v + 1] < rp[v]) atomicOr(bad, 1);
    if (tid == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(bad, 2);
    for (int64_t p = tid; p < nnz; p += stride) {
        int c = col[p];
        if (c < 0 || (int64_t)c >= n) atomicOr(bad, 4);
    }
}

// ---- expand arcs j -> i (self loops dropped) into sort keys.
// BVSS key: (new_j / sigma) << B | new_i, payload new_j % sigma.
// Transpose key (optional): new_i << B | new_j.
__global__ void k_expand(const long long *__restrict__ rp, const int *__restrict__ col, int64_t n,
                         const int *__restrict__ perm, int B, int log_sigma, unsigned long long *bkeys,
                         unsigned *bvals,
                         unsigned long long *tkeys, int *deg, unsigned long long *loops) {
    const int lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw) {
        const long long a = rp[j], b = rp[j + 1];
        const unsigned long long jn = perm ? (unsigned long long)perm[j] : (unsigned long long)j;
        int kept = 0;
        for (long long p = a + lane; p < b; p += 32) {
            const int i = col[p];
            if ((int64_t)i == j) {
                bkeys[p] = ~0ull;
                if (tkeys) tkeys[p] = ~0ull;
                atomicAdd(loops, 1ull);
                continue;
            }
            const unsigned long long in = perm ? (unsigned long long)perm[i] : (unsigned long long)i;
            bkeys[p] = ((jn >> log_sigma) << B) | in;
            bvals[p] = (unsigned)(jn & ((1ull << log_sigma) - 1ull));
            if (tkeys) tkeys[p] = (in << B) | jn;
            ++kept;
        }
        kept = warp_sum(kept);
        if (lane == 0) deg[jn] = kept;
    }
}

// run heads of a sorted key array (the first m keys are valid)
__global__ void k_heads(const unsigned long long *__restrict__ k, int64_t m, int *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += stride)
        flag[p] = (p == 0 || k[p] != k[p - 1]) ? 1 : 0;
}

// one slice per run of equal (slice set, row) keys; mask = OR of payload bits
__global__ void k_slices(const unsigned long long *__restrict__ k, const unsigned *__restrict__ v,
                         const long long *__restrict__ sidx, int64_t m, unsigned long long *skey,
                         unsigned *smask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += stride) {
        if (p != 0 && k[p] == k[p - 1]) continue;
        unsigned mask = 0;
        int64_t q = p;
        const unsigned long long key = k[p];
        while (q < m && k[q] == key) { mask |= 1u << v[q]; ++q; }
        const long long s = sidx[p];
        skey[s] = key;
        smask[s] = mask;
    }
}

// slice-set ranges [start, end) in the slice list
__global__ void k_set_ranges(const unsigned long long *__restrict__ skey, int64_t S, int B, long long *start,
                             long long *end) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += stride) {
        const unsigned long long ss = skey[s] >> B;
        if (s == 0 || (skey[s - 1] >> B) != ss) start[ss] = s;
        if (s == S - 1 || (skey[s + 1] >> B) != ss) end[ss] = s + 1;
    }
}

__global__ void k_nvss(const long long *__restrict__ start, const long long *__restrict__ end, int64_t Ns,
                       int tau, long long *nv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < Ns; s += stride)
        nv[s] = (end[s] - start[s] + tau - 1) / tau;
}

__global__ void k_real_ptrs(const long long *__restrict__ rp64, int64_t Ns, int *realPtrs, int *v2r) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= Ns; s += stride) {
        realPtrs[s] = (int)rp64[s];
        if (s < Ns)
            for (long long v = rp64[s]; v < rp64[s + 1]; ++v) v2r[v] = (int)s;
    }
}

// One thread per lane word: word g of VSS g / lanes holds the theta slices
// at slots (g / lanes) * tau + (g % lanes) * theta + c, c < theta.
__global__ void k_place(const unsigned long long *__restrict__ skey, const unsigned *__restrict__ smask,
                        const long long *__restrict__ start, const long long *__restrict__ end,
                        const int *__restrict__ realPtrs, const int *__restrict__ v2r, int64_t Nv, int B,
                        int sigma, int tau, int *rowIds, unsigned *masks) {
    const unsigned long long rmask = (B >= 64) ? ~0ull : ((1ull << B) - 1ull);
    const int theta = 32 / sigma, lanes = tau / theta;
    const unsigned fmask = sigma == 32 ? 0xFFFFFFFFu : ((1u << sigma) - 1u);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < Nv * lanes; g += stride) {
        const int64_t vss = g / lanes;
        const int l = (int)(g % lanes);
        const int ss = v2r[vss];
        const long long st = start[ss], cnt = end[ss] - st;
        const long long r0 = (long long)(vss - realPtrs[ss]) * tau + (long long)l * theta;
        unsigned word = 0;
        for (int c = 0; c < theta; ++c) {
            const long long r = r0 + c;
            int row = 0;
            if (r < cnt) {
                row = (int)(skey[st + r] & rmask);
                word |= (smask[st + r] & fmask) << (sigma * c);
            }
            rowIds[g * theta + c] = row;
        }
        masks[g] = word;
    }
}

// U_div per VSS (§4.2): mean over non-empty columns (slot position c of the
// lane words) of the population std of the row ids whose masks are nonzero.
// A warp takes 32 / lanes VSSs at once, one lane group each.
__global__ void k_udiv(const int *__restrict__ rowIds, const unsigned *__restrict__ masks, int64_t Nv, int sigma,
                       int tau, double *per_vss, unsigned long long *bits) {
    const int lane = lane_id();
    const int theta = 32 / sigma, lanes = tau / theta, G = 32 / lanes;
    const int grp = lane / lanes, l = lane % lanes;
    const unsigned fmask = sigma == 32 ? 0xFFFFFFFFu : ((1u << sigma) - 1u);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mybits = 0;
    for (int64_t v0 = gw * G; v0 < Nv; v0 += nw * G) {
        const int64_t v = v0 + grp;
        const bool valid = v < Nv;
        const int64_t wi = v * lanes + l;
        const unsigned m = valid ? masks[wi] : 0u;
        mybits += __popc(m);
        double tot = 0.0;
        int ncols = 0;
        for (int c = 0; c < theta; ++c) {
            const bool ok = ((m >> (sigma * c)) & fmask) != 0;
            const double x = ok ? (double)rowIds[wi * theta + c] : 0.0;
            int cnt = ok ? 1 : 0;
            double sx = x;
            for (int o = lanes / 2; o > 0; o >>= 1) {
                cnt += __shfl_xor_sync(FULL_MASK, cnt, o, lanes);
                sx += __shfl_xor_sync(FULL_MASK, sx, o, lanes);
            }
            // every lane takes part in the shuffles; empty columns add nothing
            const double mean = cnt ? sx / (double)cnt : 0.0;
            const double d = ok ? (x - mean) : 0.0;
            double sq = d * d;
            for (int o = lanes / 2; o > 0; o >>= 1) sq += __shfl_xor_sync(FULL_MASK, sq, o, lanes);
            if (cnt) {
                tot += sqrt(sq / (double)cnt);
                ++ncols;
            }
        }
        if (valid && l == 0) per_vss[v] = ncols ? tot / (double)ncols : 0.0;
    }
    mybits = warp_sum(mybits);
    if (lane == 0 && mybits) atomicAdd(bits, mybits);
}

// fixed-order sum of doubles: block b sums chunk b with a tree
__global__ void k_dsum_partial(const double *__restrict__ x, int64_t n, int64_t chunk, double *part) {
    __shared__ double sh[TB];
    const int64_t a = (int64_t)blockIdx.x * chunk, e = (a + chunk < n) ? a + chunk : n;
    double acc = 0.0;
    for (int64_t i = a + threadIdx.x; i < e; i += TB) acc += x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = TB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// CSR from sorted transpose keys: row = key >> B, col = key & mask
__global__ void k_tcsr_rows(const unsigned long long *__restrict__ k, int64_t m, int B, long long *rp,
                            int *col) {
    const unsigned long long rmask = (1ull << B) - 1ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += stride) {
        const unsigned long long key = k[p];
        const long long row = (long long)(key >> B);
        col[p] = (int)(key & rmask);
        if (p == 0) {
            for (long long r = 0; r <= row; ++r) rp[r] = 0;
        } else {
            const long long prow = (long long)(k[p - 1] >> B);
            for (long long r = prow + 1; r <= row; ++r) rp[r] = p;
        }
    }
}
__global__ void k_tcsr_tail(const unsigned long long *__restrict__ k, int64_t m, int B, int64_t n,
                            long long *rp) {
    const long long last = m ? (long long)(k[m - 1] >> B) : -1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = last + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += stride)
        rp[r] = m;
}

// Bottom-up rows sorted by descending degree of the in-neighbour (hubs are
// the likeliest frontier members, so they are probed first; levels do not
// depend on the probe order).  key = row << 31 | (2^31 - 1 - degree).
__global__ void k_bu_keys(const long long *__restrict__ rp, const int *__restrict__ col, int64_t n,
                          const int *__restrict__ deg, unsigned long long *keys, unsigned *vals) {
    const int lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw)
        for (long long p = rp[j] + lane; p < rp[j + 1]; p += 32) {
            const int v = col[p];
            keys[p] = ((unsigned long long)j << 31) | (unsigned long long)(0x7FFFFFFF - deg[v]);
            vals[p] = (unsigned)v;
        }
}

// head[u] = the first four in-neighbours of u (-1 where the row is shorter)
__global__ void k_bu_head(const long long *__restrict__ rp, const int *__restrict__ col, int64_t n, int4 *head) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const long long a = rp[u], d = rp[u + 1] - a;
        head[u] = make_int4(d > 0 ? col[a] : -1, d > 1 ? col[a + 1] : -1, d > 2 ? col[a + 2] : -1,
                            d > 3 ? col[a + 3] : -1);
    }
}

__global__ void k_inverse_perm(const int *__restrict__ new_of_old, int64_t n, int *old_of_new) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        old_of_new[new_of_old[v]] = (int)v;
}

struct TmpPool {
    cudaStream_t st;
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, count * sizeof(T) + 16, st);
        if (e != cudaSuccess) { err = e; return nullptr; }
        ptrs.push_back(p);
        return (T *)p;
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) { cudaFreeAsync(q, st); q = nullptr; }
    }
    ~TmpPool() {
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace

#define BUILD_TRY(expr)                                                          \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess) {                                                 \
            blest_internal_record_cuda_error(_e, #expr, __FILE__, __LINE__);     \
            return (_e == cudaErrorMemoryAllocation) ? BLEST_ERR_OOM : BLEST_ERR_CUDA; \
        }                                                                        \
    } while (0)
#define POOL_CHECK(pool) BUILD_TRY((pool).err)

blest_status build_graph(blest_graph *h, const int64_t *row_ptr, const int32_t *col_idx,
                         const blest_build_opts *o) {
    cudaStream_t st = h->stream;
    const int64_t n = h->n;
    // row_ptr[n] tells the arc count
    int64_t nnz_in = 0;
    BUILD_TRY(cudaMemcpy(&nnz_in, row_ptr + n, sizeof(int64_t), cudaMemcpyDefault));
    if (nnz_in < 0 || nnz_in >= ((int64_t)1 << 40)) return BLEST_ERR_INVALID;

    cudaEvent_t e0, e1;
    BUILD_TRY(cudaEventCreate(&e0));
    BUILD_TRY(cudaEventCreate(&e1));
    BUILD_TRY(cudaEventRecord(e0, st));

    TmpPool pool{st};
    long long *rp_in = nullptr;
    int *col_in = nullptr;
    blest_status bs;
    if ((bs = dev_alloc_t(h, &rp_in, (size_t)n + 1)) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &col_in, (size_t)(nnz_in > 0 ? nnz_in : 1))) != BLEST_OK) return bs;
    BUILD_TRY(cudaMemcpyAsync(rp_in, row_ptr, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDefault, st));
    if (nnz_in > 0)
        BUILD_TRY(cudaMemcpyAsync(col_in, col_idx, (size_t)nnz_in * sizeof(int32_t), cudaMemcpyDefault, st));

    int *d_bad = pool.get<int>(1);
    POOL_CHECK(pool);
    BUILD_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    k_validate<<<grid_for(n > nnz_in ? n : nnz_in, TB, 8192), TB, 0, st>>>(rp_in, col_in, n, nnz_in, d_bad);
    int bad = 0;
    BUILD_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    BUILD_TRY(cudaStreamSynchronize(st));
    if (bad) return BLEST_ERR_INVALID;

    // ---- reordering (§4): new_of_old permutation on the device
    int *perm = nullptr;
    h->reorder = BLEST_REORDER_NONE;
    if (o->reorder != BLEST_REORDER_NONE) {
        int applied = BLEST_REORDER_NONE;
        if ((bs = dev_alloc_t(h, &perm, (size_t)n)) != BLEST_OK) return bs;
        bs = reorder_graph(h, rp_in, col_in, n, nnz_in, o, perm, &applied);
        if (bs != BLEST_OK) return bs;
        h->reorder = applied;
        if ((bs = dev_alloc_t(h, &h->g.old_of_new, (size_t)n)) != BLEST_OK) return bs;
        k_inverse_perm<<<grid_for(n), TB, 0, st>>>(perm, n, h->g.old_of_new);
        h->g.new_of_old = perm;
    }

    const int B = ceil_log2_i64(n) > 0 ? ceil_log2_i64(n) : 1;
    const int sigma = h->sigma, tau = h->tau, theta = 32 / sigma, lanes = tau / theta;
    const int log_sigma = sigma == 8 ? 3 : (sigma == 16 ? 4 : 5);
    const int64_t Ns = (n + sigma - 1) / sigma;
    const int SB = ceil_log2_i64(Ns) > 0 ? ceil_log2_i64(Ns) : 1;
    const bool need_t = h->directed || perm != nullptr;
    const int64_t M = nnz_in;

    unsigned long long *bk = pool.get<unsigned long long>((size_t)M + 1);
    unsigned *bv = pool.get<unsigned>((size_t)M + 1);
    unsigned long long *tk = need_t ? pool.get<unsigned long long>((size_t)M + 1) : nullptr;
    unsigned long long *d_loops = pool.get<unsigned long long>(1);
    int *deg = nullptr;
    POOL_CHECK(pool);
    if ((bs = dev_alloc_t(h, &deg, (size_t)n)) != BLEST_OK) return bs;
    h->g.deg = deg;
    BUILD_TRY(cudaMemsetAsync(d_loops, 0, sizeof(unsigned long long), st));
    BUILD_TRY(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int), st));
    k_expand<<<grid_for(n * 32, TB, 1 << 16), TB, 0, st>>>(rp_in, col_in, n, perm, B, log_sigma, bk, bv, tk, deg,
                                                            d_loops);
    BUILD_TRY(cudaGetLastError());
    unsigned long long loops = 0;
    BUILD_TRY(cudaMemcpyAsync(&loops, d_loops, sizeof(loops), cudaMemcpyDeviceToHost, st));
    BUILD_TRY(cudaStreamSynchronize(st));
    const int64_t m = M - (int64_t)loops;   // valid (non-loop) arcs; loops sort last

    // ---- sort BVSS keys (slice set, row)
    {
        unsigned long long *kalt = pool.get<unsigned long long>((size_t)M + 1);
        unsigned *valt = pool.get<unsigned>((size_t)M + 1);
        long long *hist = pool.get<long long>(radix_hist_elems(M));
        long long *stmp = pool.get<long long>(scan_tmp_elems((int64_t)radix_hist_elems(M)) + 16);
        POOL_CHECK(pool);
        BUILD_TRY(radix_sort_u64(bk, bv, kalt, valt, M, SB + B + 1, hist, stmp, st));  // +1: loops sort last
        if (tk) BUILD_TRY(radix_sort_u64(tk, nullptr, kalt, nullptr, M, 2 * B + 1, hist, stmp, st));
        pool.release(kalt);
        pool.release(valt);
        pool.release(hist);
        pool.release(stmp);
    }

    // ---- slices: one per run of equal keys
    int *flag = pool.get<int>((size_t)m + 1);
    long long *sidx = pool.get<long long>((size_t)m + 2);
    long long *stmp = pool.get<long long>(scan_tmp_elems(m > Ns ? m : Ns) + 16);
    POOL_CHECK(pool);
    k_heads<<<grid_for(m, TB, 1 << 16), TB, 0, st>>>(bk, m, flag);
    BUILD_TRY(scan_exclusive_i32_to_i64(flag, sidx, m, stmp, st));
    long long S = 0;
    BUILD_TRY(cudaMemcpyAsync(&S, sidx + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    BUILD_TRY(cudaStreamSynchronize(st));
    h->num_slices = S;
    unsigned long long *skey = pool.get<unsigned long long>((size_t)S + 1);
    unsigned *smask = pool.get<unsigned>((size_t)S + 1);
    long long *start = pool.get<long long>((size_t)Ns + 1);
    long long *end = pool.get<long long>((size_t)Ns + 1);
    long long *nv = pool.get<long long>((size_t)Ns + 2);
    POOL_CHECK(pool);
    k_slices<<<grid_for(m, TB, 1 << 16), TB, 0, st>>>(bk, bv, sidx, m, skey, smask);
    BUILD_TRY(cudaMemsetAsync(start, 0, ((size_t)Ns + 1) * sizeof(long long), st));
    BUILD_TRY(cudaMemsetAsync(end, 0, ((size_t)Ns + 1) * sizeof(long long), st));
    k_set_ranges<<<grid_for(S, TB, 1 << 16), TB, 0, st>>>(skey, S, B, start, end);
    k_nvss<<<grid_for(Ns, TB, 1 << 16), TB, 0, st>>>(start, end, Ns, tau, nv);
    BUILD_TRY(scan_exclusive_i64(nv, nv, Ns, stmp, st));
    long long Nv = 0;
    BUILD_TRY(cudaMemcpyAsync(&Nv, nv + Ns, sizeof(long long), cudaMemcpyDeviceToHost, st));
    BUILD_TRY(cudaStreamSynchronize(st));
    if (Nv * lanes >= ((long long)1 << 31)) return BLEST_ERR_UNSUPPORTED;   // lane words (64-bit slot indexing)
    h->Ns = Ns;
    h->Nv = Nv;
    if ((bs = dev_alloc_t(h, &h->g.realPtrs, (size_t)Ns + 1)) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &h->g.v2r, (size_t)(Nv > 0 ? Nv : 1))) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &h->g.rowIds, (size_t)(Nv > 0 ? Nv : 1) * tau)) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &h->g.masks, (size_t)(Nv > 0 ? Nv : 1) * lanes)) != BLEST_OK) return bs;
    k_real_ptrs<<<grid_for(Ns + 1, TB, 1 << 16), TB, 0, st>>>(nv, Ns, h->g.realPtrs, h->g.v2r);
    if (Nv > 0)
        k_place<<<grid_for(Nv * lanes, TB, 1 << 16), TB, 0, st>>>(skey, smask, start, end, h->g.realPtrs,
                                                                     h->g.v2r, Nv, B, sigma, tau, h->g.rowIds,
                                                                     h->g.masks);
    BUILD_TRY(cudaGetLastError());

    // ---- U_div and distinct arc count
    {
        double *pv = pool.get<double>((size_t)(Nv > 0 ? Nv : 1));
        unsigned long long *bits = pool.get<unsigned long long>(1);
        const int64_t chunk = 1 << 16;
        const int64_t nparts = (Nv + chunk - 1) / chunk > 0 ? (Nv + chunk - 1) / chunk : 1;
        double *part = pool.get<double>((size_t)nparts);
        double *one = pool.get<double>(1);
        POOL_CHECK(pool);
        BUILD_TRY(cudaMemsetAsync(bits, 0, sizeof(unsigned long long), st));
        if (Nv > 0) {
            k_udiv<<<grid_for(Nv * lanes, TB, 1 << 16), TB, 0, st>>>(h->g.rowIds, h->g.masks, Nv, sigma, tau, pv,
                                                                        bits);
            k_dsum_partial<<<(unsigned)nparts, TB, 0, st>>>(pv, Nv, chunk, part);
            k_dsum_partial<<<1, TB, 0, st>>>(part, nparts, nparts, one);
        } else {
            BUILD_TRY(cudaMemsetAsync(one, 0, sizeof(double), st));
        }
        double sum = 0.0;
        unsigned long long nb = 0;
        BUILD_TRY(cudaMemcpyAsync(&sum, one, sizeof(double), cudaMemcpyDeviceToHost, st));
        BUILD_TRY(cudaMemcpyAsync(&nb, bits, sizeof(nb), cudaMemcpyDeviceToHost, st));
        BUILD_TRY(cudaStreamSynchronize(st));
        h->udiv = Nv > 0 ? sum / (double)Nv : 0.0;
        h->nnz = (int64_t)nb;
    }

    // ---- in-neighbour CSR for bottom-up levels
    if (!need_t) {
        h->g.rp = rp_in;
        h->g.col = col_in;
    } else {
        long long *rp = nullptr;
        int *col = nullptr;
        if ((bs = dev_alloc_t(h, &rp, (size_t)n + 1)) != BLEST_OK) return bs;
        if ((bs = dev_alloc_t(h, &col, (size_t)(m > 0 ? m : 1))) != BLEST_OK) return bs;
        if (m > 0) k_tcsr_rows<<<grid_for(m, TB, 1 << 16), TB, 0, st>>>(tk, m, B, rp, col);
        k_tcsr_tail<<<grid_for(n + 1, TB, 1 << 16), TB, 0, st>>>(tk, m, B, n, rp);
        h->g.rp = rp;
        h->g.col = col;
    }
    BUILD_TRY(cudaGetLastError());
    // rows by descending neighbour degree, and the 4-neighbour head of each row
    {
        long long nb = 0;
        BUILD_TRY(cudaMemcpyAsync(&nb, h->g.rp + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
        BUILD_TRY(cudaStreamSynchronize(st));
        if (nb > 0) {
            unsigned long long *kk = pool.get<unsigned long long>((size_t)nb + 1);
            unsigned long long *ka = pool.get<unsigned long long>((size_t)nb + 1);
            unsigned *vv = pool.get<unsigned>((size_t)nb + 1);
            unsigned *va = pool.get<unsigned>((size_t)nb + 1);
            long long *hist = pool.get<long long>(radix_hist_elems(nb));
            long long *stmp2 = pool.get<long long>(scan_tmp_elems((int64_t)radix_hist_elems(nb)) + 16);
            int *colbu = nullptr;
            POOL_CHECK(pool);
            if ((bs = dev_alloc_t(h, &colbu, (size_t)nb)) != BLEST_OK) return bs;
            k_bu_keys<<<grid_for(n * 32, TB, 1 << 16), TB, 0, st>>>(h->g.rp, h->g.col, n, deg, kk, vv);
            BUILD_TRY(radix_sort_u64(kk, vv, ka, va, nb, B + 31, hist, stmp2, st));
            BUILD_TRY(cudaMemcpyAsync(colbu, vv, (size_t)nb * 4, cudaMemcpyDeviceToDevice, st));
            h->g.col = colbu;
            pool.release(kk); pool.release(ka); pool.release(vv); pool.release(va);
            pool.release(hist); pool.release(stmp2);
        }
        if ((bs = dev_alloc_t(h, &h->g.head, (size_t)n)) != BLEST_OK) return bs;
        k_bu_head<<<grid_for(n, TB, 1 << 16), TB, 0, st>>>(h->g.rp, h->g.col, n, h->g.head);
        BUILD_TRY(cudaGetLastError());
    }
    BUILD_TRY(cudaEventRecord(e1, st));
    BUILD_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return BLEST_OK;
}
