// Batched BFS over many small graphs in one persistent launch.
//
// blest_build_many lays the graphs out as one disjoint union whose per-graph
// vertex ranges are padded to multiples of sigma = 8, so no slice set spans
// two graphs, and builds one BVSS (§3.1) for the union.  blest_bfs_many runs
// one BFS per graph: a CTA takes the next graph from an atomic counter over
// the graphs sorted by size, largest first (longest-processing-time order),
// and runs Algorithm 2 (eager push over the graph's VSS queue) with the
// graph's visited and frontier bitvectors in shared memory and CTA-local
// barriers between levels -- no grid-wide synchronisation at all.  The launch
// (source upload, counter reset, kernel) is captured once in a CUDA graph
// and replayed.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "msbfs.h"

struct ManyGraphs {
    int G = 0;
    int max_n = 0;          // largest graph (vertices)
    int max_words = 0;      // ceil(padded max_n / 32)
    int max_nv = 0;         // most VSSs of one graph
    int *pvo = nullptr;     // padded vertex offset per graph (union ids)
    int *nv = nullptr;      // vertices per graph
    long long *vo = nullptr;  // caller's vertex offset per graph
    int *order = nullptr;   // graphs by decreasing size
    int *counter = nullptr;
    int *qscratch = nullptr;
    int *d_src = nullptr;
    int *h_src = nullptr;   // pinned
    int grid = 0;
    size_t smem = 0;
    int block = 256;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    void *exec_out = nullptr;
    cudaStream_t exec_stream = nullptr;
    std::vector<long long> vo_host;
};

namespace {

constexpr int MANY_BLOCK = 256;

struct ManyParams {
    int G;
    const int *__restrict__ rowIds;   // sigma = 8, tau = 128: one int4 per lane word
    const unsigned *__restrict__ masks;
    const int *__restrict__ realPtrs;
    const int *__restrict__ v2r;
    const int *__restrict__ pvo;
    const int *__restrict__ nv;
    const long long *__restrict__ vo;
    const int *__restrict__ order;
    const int *__restrict__ src;
    int *counter;
    int *qscratch;
    int qcap;
    int words;
    int *levels;
    int tc;
};

__device__ __forceinline__ unsigned hits_cc_m(unsigned m, unsigned alpha) {
    const unsigned x = m & (alpha * 0x01010101u);
    return (unsigned)((x & 0xFFu) != 0) | ((unsigned)((x & 0xFF00u) != 0) << 1) |
           ((unsigned)((x & 0xFF0000u) != 0) << 2) | ((unsigned)((x >> 24) != 0) << 3);
}
__device__ __forceinline__ unsigned hits_tc_m(unsigned m, unsigned alpha, unsigned bsel) {
    const unsigned fb = alpha * bsel;
    int d0, d1, d2, d3;
    asm volatile("mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
                 : "=r"(d0), "=r"(d1) : "r"(m & 0xFFFFu), "r"(fb), "r"(0), "r"(0));
    asm volatile("mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
                 : "=r"(d2), "=r"(d3) : "r"(m >> 16), "r"(fb), "r"(0), "r"(0));
    return (unsigned)(d0 != 0) | ((unsigned)(d1 != 0) << 1) | ((unsigned)(d2 != 0) << 2) |
           ((unsigned)(d3 != 0) << 3);
}

__global__ void __launch_bounds__(MANY_BLOCK) k_many(ManyParams P) {
    extern __shared__ unsigned sm[];
    unsigned *V = sm;                    // visited bits (local ids)
    unsigned *Fb[2] = {sm + P.words, sm + 2 * P.words};
    __shared__ int s_g, s_qlen[2];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned bsel = (lane % 9 == 0) ? 1u : ((lane % 9 == 4) ? 256u : 0u);
    int *Qb[2] = {P.qscratch + (size_t)blockIdx.x * 2 * P.qcap, P.qscratch + (size_t)blockIdx.x * 2 * P.qcap + P.qcap};

    for (;;) {
        if (threadIdx.x == 0) s_g = atomicAdd(P.counter, 1);
        __syncthreads();
        const int gi = s_g;
        if (gi >= P.G) break;
        const int gidx = P.order[gi];
        const int n = P.nv[gidx];
        const int base = P.pvo[gidx];          // union id of local vertex 0 (multiple of 8)
        const long long out0 = P.vo[gidx];
        const int words = (n + 31) >> 5;
        for (int i = threadIdx.x; i < words; i += blockDim.x) { V[i] = 0u; Fb[0][i] = 0u; Fb[1][i] = 0u; }
        for (int i = threadIdx.x; i < n; i += blockDim.x) P.levels[out0 + i] = -1;
        if (threadIdx.x == 0) { s_qlen[0] = 0; s_qlen[1] = 0; }
        __syncthreads();
        const int s = P.src[gidx];
        if (s >= 0 && s < n) {
            const int ss = (base + s) >> 3;
            const int a = __ldg(&P.realPtrs[ss]), e = __ldg(&P.realPtrs[ss + 1]);
            for (int k = threadIdx.x; k < e - a; k += blockDim.x) Qb[0][k] = a + k;
            if (threadIdx.x == 0) {
                V[s >> 5] = 1u << (s & 31);
                Fb[0][s >> 5] = 1u << (s & 31);
                P.levels[out0 + s] = 0;
                s_qlen[0] = e - a;
            }
        }
        __syncthreads();
        int cur = 0;
        for (int ell = 1;; ++ell) {
            const int qlen = s_qlen[cur];
            if (qlen == 0) break;
            const unsigned char *Fc = reinterpret_cast<const unsigned char *>(Fb[cur]);
            unsigned *Fn = Fb[cur ^ 1];
            int *Qn = Qb[cur ^ 1];
            for (int w = wid; w < qlen; w += nw) {
                const int vss = Qb[cur][w];
                const int ls = __ldg(&P.v2r[vss]) - (base >> 3);
                const int4 r = __ldg(reinterpret_cast<const int4 *>(P.rowIds) + (size_t)vss * 32 + lane);
                const unsigned m = __ldg(&P.masks[(size_t)vss * 32 + lane]);
                const unsigned alpha = Fc[ls];
                const unsigned hits = P.tc ? hits_tc_m(m, alpha, bsel) : hits_cc_m(m, alpha);
                int want_len[4] = {0, 0, 0, 0}, want_a[4] = {0, 0, 0, 0};
                int tot = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (hits >> c & 1u) {
                        const int u = (c == 0 ? r.x : (c == 1 ? r.y : (c == 2 ? r.z : r.w))) - base;
                        const unsigned bit = 1u << (u & 31);
                        if (!(V[u >> 5] & bit)) {
                            const unsigned old = atomicOr(&Fn[u >> 5], bit);
                            if (!(old & bit)) {
                                atomicOr(&V[u >> 5], bit);
                                P.levels[out0 + u] = ell;
                                if (((old >> (u & 24)) & 0xFFu) == 0) {
                                    const int so = (base + u) >> 3;
                                    want_a[c] = __ldg(&P.realPtrs[so]);
                                    want_len[c] = __ldg(&P.realPtrs[so + 1]) - want_a[c];
                                    tot += want_len[c];
                                }
                            }
                        }
                    }
                }
                // warp-aggregated append to the next queue
                const int incl = warp_incl_scan(tot);
                int qb = 0;
                if (lane == 31 && incl) qb = atomicAdd(&s_qlen[cur ^ 1], incl);
                qb = __shfl_sync(FULL_MASK, qb, 31) + incl - tot;
                // each lane appends its own ranges: hub slice sets of graphs this
                // small span few VSSs, and a warp-wide pass measured slower here
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    for (int k = 0; k < want_len[c]; ++k) Qn[qb++] = want_a[c] + k;
            }
            __syncthreads();
            // the current frontier becomes the next level's (cleared) target
            unsigned *Fo = Fb[cur];
            for (int i = threadIdx.x; i < words; i += blockDim.x) Fo[i] = 0u;
            if (threadIdx.x == 0) s_qlen[cur] = 0;
            cur ^= 1;
            __syncthreads();
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------- build
__global__ void k_union_csr(const long long *__restrict__ vtx_off, const long long *__restrict__ edge_off,
                            const long long *__restrict__ rp_local, const int *__restrict__ col_local,
                            const int *__restrict__ pvo, int G, long long *rp_u, int *col_u, long long n_u) {
    for (int i = blockIdx.x; i < G; i += gridDim.x) {
        const long long v0 = vtx_off[i], n = vtx_off[i + 1] - v0;
        const long long e0 = edge_off[i], e1 = edge_off[i + 1];
        const long long pb = pvo[i];
        const long long pn = (i + 1 < G) ? (long long)pvo[i + 1] : n_u;
        for (long long v = threadIdx.x; v < pn - pb; v += blockDim.x)
            rp_u[pb + v] = (v < n) ? e0 + rp_local[v0 + i + v] : e1;
        for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) col_u[e] = col_local[e] + (int)pb;
        if (i == G - 1 && threadIdx.x == 0) rp_u[n_u] = e1;
    }
}

extern "C" blest_status blest_build_many(int32_t g, const int64_t *vtx_off, const int64_t *edge_off,
                                         const int64_t *row_ptr, const int32_t *col_idx_local,
                                         const blest_build_opts *opts, blest_handle *out) {
    if (!out || g < 1 || !vtx_off || !edge_off || !row_ptr || !col_idx_local) return BLEST_ERR_INVALID;
    *out = nullptr;
    std::vector<long long> vo((size_t)g + 1), eo((size_t)g + 1);
    if (cudaMemcpy(vo.data(), vtx_off, ((size_t)g + 1) * 8, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(eo.data(), edge_off, ((size_t)g + 1) * 8, cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (vo[0] != 0 || eo[0] != 0) return BLEST_ERR_INVALID;
    std::vector<int> pvo((size_t)g), nvv((size_t)g);
    long long acc = 0;
    int max_n = 0;
    for (int i = 0; i < g; ++i) {
        const long long n = vo[(size_t)i + 1] - vo[(size_t)i];
        if (n < 1 || n > 500000 || eo[(size_t)i + 1] < eo[(size_t)i]) return BLEST_ERR_INVALID;
        pvo[(size_t)i] = (int)acc;
        nvv[(size_t)i] = (int)n;
        max_n = std::max(max_n, (int)n);
        acc += (n + 7) / 8 * 8;
        if (acc >= ((long long)1 << 31) - 64) return BLEST_ERR_UNSUPPORTED;
    }
    const long long n_u = acc;
    const long long m = eo[(size_t)g];
    // union CSR on the device
    long long *d_vo = nullptr, *d_eo = nullptr, *d_rpl = nullptr, *d_rpu = nullptr;
    int *d_coll = nullptr, *d_colu = nullptr, *d_pvo = nullptr;
    const long long rpl_len = vo[(size_t)g] + g;
    bool ok = cudaMalloc(&d_vo, ((size_t)g + 1) * 8) == cudaSuccess &&
              cudaMalloc(&d_eo, ((size_t)g + 1) * 8) == cudaSuccess &&
              cudaMalloc(&d_rpl, (size_t)rpl_len * 8) == cudaSuccess &&
              cudaMalloc(&d_coll, (size_t)(m > 0 ? m : 1) * 4) == cudaSuccess &&
              cudaMalloc(&d_rpu, ((size_t)n_u + 1) * 8) == cudaSuccess &&
              cudaMalloc(&d_colu, (size_t)(m > 0 ? m : 1) * 4) == cudaSuccess &&
              cudaMalloc(&d_pvo, (size_t)g * 4) == cudaSuccess;
    blest_status st = BLEST_OK;
    if (!ok) st = BLEST_ERR_OOM;
    if (st == BLEST_OK) {
        cudaMemcpy(d_vo, vo.data(), ((size_t)g + 1) * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(d_eo, eo.data(), ((size_t)g + 1) * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(d_rpl, row_ptr, (size_t)rpl_len * 8, cudaMemcpyDefault);
        if (m > 0) cudaMemcpy(d_coll, col_idx_local, (size_t)m * 4, cudaMemcpyDefault);
        cudaMemcpy(d_pvo, pvo.data(), (size_t)g * 4, cudaMemcpyHostToDevice);
        k_union_csr<<<std::min(g, 65535), 256>>>(d_vo, d_eo, d_rpl, d_coll, d_pvo, g, d_rpu, d_colu, n_u);
        if (cudaDeviceSynchronize() != cudaSuccess) st = BLEST_ERR_CUDA;
    }
    cudaFree(d_vo); cudaFree(d_eo); cudaFree(d_rpl); cudaFree(d_coll); cudaFree(d_pvo);
    blest_handle h = nullptr;
    if (st == BLEST_OK) {
        blest_build_opts o;
        blest_default_opts(&o);
        if (opts) o = *opts;
        o.reorder = BLEST_REORDER_NONE;  // the union keeps each graph's own numbering
        o.directed = 0;
        o.probe_switch = 0;
        if ((o.sigma != 0 && o.sigma != 8) || (o.tau != 0 && o.tau != 128)) st = BLEST_ERR_UNSUPPORTED;
        else st = blest_build(n_u, (const int64_t *)d_rpu, d_colu, &o, &h);
    }
    cudaFree(d_rpu);
    cudaFree(d_colu);
    if (st != BLEST_OK) return st;

    ManyGraphs *mg = new ManyGraphs();
    mg->G = g;
    mg->max_n = max_n;
    mg->max_words = (max_n + 31) / 32 + 1;
    mg->vo_host.assign(vo.begin(), vo.end());
    // VSSs per graph from realPtrs at the graph's slice-set boundaries
    std::vector<int> rp((size_t)h->Ns + 1);
    cudaMemcpy(rp.data(), h->g.realPtrs, ((size_t)h->Ns + 1) * 4, cudaMemcpyDeviceToHost);
    int max_nv = 1;
    for (int i = 0; i < g; ++i) {
        const long long s0 = pvo[(size_t)i] / 8;
        const long long s1 = (i + 1 < g) ? pvo[(size_t)i + 1] / 8 : n_u / 8;
        max_nv = std::max(max_nv, rp[(size_t)s1] - rp[(size_t)s0]);
    }
    mg->max_nv = max_nv;
    std::vector<int> order((size_t)g);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nvv[(size_t)a] > nvv[(size_t)b]; });
    std::vector<long long> vo_g(vo.begin(), vo.begin() + g);
    if ((st = dev_alloc_t(h, &mg->pvo, (size_t)g)) != BLEST_OK ||
        (st = dev_alloc_t(h, &mg->nv, (size_t)g)) != BLEST_OK ||
        (st = dev_alloc_t(h, &mg->vo, (size_t)g)) != BLEST_OK ||
        (st = dev_alloc_t(h, &mg->order, (size_t)g)) != BLEST_OK ||
        (st = dev_alloc_t(h, &mg->counter, 1)) != BLEST_OK ||
        (st = dev_alloc_t(h, &mg->d_src, (size_t)g)) != BLEST_OK) {
        delete mg;
        blest_destroy(h);
        return st;
    }
    cudaMemcpy(mg->pvo, pvo.data(), (size_t)g * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(mg->nv, nvv.data(), (size_t)g * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(mg->vo, vo_g.data(), (size_t)g * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(mg->order, order.data(), (size_t)g * 4, cudaMemcpyHostToDevice);
    mg->smem = (size_t)3 * mg->max_words * 4;
    if (mg->smem > 200 * 1024) { delete mg; blest_destroy(h); return BLEST_ERR_UNSUPPORTED; }
    cudaFuncSetAttribute(k_many, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mg->smem);
    int per = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_many, MANY_BLOCK, mg->smem);
    mg->grid = std::max(1, per) * sms;
    if ((st = dev_alloc_t(h, &mg->qscratch, (size_t)mg->grid * 2 * mg->max_nv)) != BLEST_OK) {
        delete mg; blest_destroy(h); return st;
    }
    if (cudaMallocHost((void **)&mg->h_src, (size_t)g * 4) != cudaSuccess) { delete mg; blest_destroy(h); return BLEST_ERR_OOM; }
    h->many = mg;
    *out = h;
    return BLEST_OK;
}

void many_release(blest_graph *h) {
    ManyGraphs *mg = h->many;
    if (!mg) return;
    if (mg->exec) cudaGraphExecDestroy(mg->exec);
    if (mg->graph) cudaGraphDestroy(mg->graph);
    if (mg->h_src) cudaFreeHost(mg->h_src);
    delete mg;
    h->many = nullptr;
}

static blest_status many_capture(blest_graph *h, int32_t *levels_dev) {
    ManyGraphs *mg = h->many;
    if (mg->exec && mg->exec_out == levels_dev && mg->exec_stream == h->stream) return BLEST_OK;
    if (mg->exec) { cudaGraphExecDestroy(mg->exec); mg->exec = nullptr; }
    if (mg->graph) { cudaGraphDestroy(mg->graph); mg->graph = nullptr; }
    ManyParams P;
    memset(&P, 0, sizeof P);
    P.G = mg->G;
    P.rowIds = h->g.rowIds;
    P.masks = h->g.masks;
    P.realPtrs = h->g.realPtrs;
    P.v2r = h->g.v2r;
    P.pvo = mg->pvo;
    P.nv = mg->nv;
    P.vo = mg->vo;
    P.order = mg->order;
    P.src = mg->d_src;
    P.counter = mg->counter;
    P.qscratch = mg->qscratch;
    P.qcap = mg->max_nv;
    P.words = mg->max_words;
    P.levels = levels_dev;
    P.tc = h->engine_tc;
    cudaStream_t cs = h->stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BLEST_ERR_CUDA;
    cudaMemcpyAsync(mg->d_src, mg->h_src, (size_t)mg->G * 4, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(mg->counter, 0, sizeof(int), cs);
    k_many<<<mg->grid, MANY_BLOCK, mg->smem, cs>>>(P);
    if (cudaStreamEndCapture(cs, &mg->graph) != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaGraphInstantiate(&mg->exec, mg->graph, 0) != cudaSuccess) return BLEST_ERR_CUDA;
    mg->exec_out = levels_dev;
    mg->exec_stream = h->stream;
    return BLEST_OK;
}

extern "C" blest_status blest_bfs_many(blest_handle h, const int32_t *sources, int32_t *levels) {
    if (!h || !h->many || !sources || !levels) return BLEST_ERR_INVALID;
    ManyGraphs *mg = h->many;
    // the previous replay may still read the pinned source buffer
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaMemcpy(mg->h_src, sources, (size_t)mg->G * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    for (int i = 0; i < mg->G; ++i)
        if (mg->h_src[i] < 0 || (long long)mg->h_src[i] >= mg->vo_host[(size_t)i + 1] - mg->vo_host[(size_t)i])
            return BLEST_ERR_INVALID;
    const long long total = mg->vo_host[(size_t)mg->G];
    const bool dev = is_device_ptr(levels);
    blest_status st = BLEST_OK;
    int32_t *target = levels;
    if (!dev) {
        if (!h->w.stage || h->w.stage_count < (size_t)total) {
            void *p = nullptr;
            if ((st = dev_alloc(h, &p, (size_t)total * 4 + 16)) != BLEST_OK) return st;
            h->w.stage = (int32_t *)p;
            h->w.stage_count = (size_t)total;
        }
        target = h->w.stage;
    }
    if ((st = many_capture(h, target)) != BLEST_OK) return st;
    if (cudaGraphLaunch(mg->exec, h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    if (!dev) {
        if (cudaMemcpyAsync(levels, target, (size_t)total * 4, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
            return BLEST_ERR_CUDA;
    }
    if (dev && h->async) return BLEST_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    return BLEST_OK;
}
