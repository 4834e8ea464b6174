// C ABI entry points (include/blest.h): handle lifetime, argument checks,
// host/device output handling and device-status reporting.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "handle.h"
#include "mlp.h"
#include "msbfs.h"

static thread_local char g_last_cuda_error[512];

extern "C" void blest_internal_record_cuda_error(cudaError_t e, const char *expr, const char *file, int line) {
    snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s:%d %s -> %s", file, line, expr,
             cudaGetErrorString(e));
    if (getenv("BLEST_VERBOSE")) fprintf(stderr, "blest: %s\n", g_last_cuda_error);
}

extern "C" const char *blest_last_cuda_error(void) { return g_last_cuda_error; }

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

blest_status dev_alloc(blest_graph *h, void **p, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? BLEST_ERR_OOM : BLEST_ERR_CUDA;
    }
    h->allocations.push_back(q);
    h->device_bytes += (int64_t)bytes;
    *p = q;
    return BLEST_OK;
}

static void free_all(blest_graph *h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *p : h->allocations) cudaFree(p);
    h->allocations.clear();
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    msbfs_release(h);
    many_release(h);
}

extern "C" void blest_default_opts(blest_build_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->reorder = BLEST_REORDER_NONE;
    o->sigma = 8;
    o->directed = 0;
    o->jaccard_window = 65536;
    o->probe_switch = 1;
    o->engine_tc = 0;
    o->eta = 10.f;
    o->udiv_threshold = 25000.0;
    o->timeout_ms = 5000;
    o->block_threads = 512;
    o->vss_batch = 2;
}

static blest_status finish_call(blest_graph *h, bool must_sync) {
    cudaError_t e = cudaMemcpyAsync(h->h_ctl, h->w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return BLEST_ERR_CUDA;
    if (!must_sync && h->async) return BLEST_OK;
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        blest_internal_record_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
        return BLEST_ERR_CUDA;
    }
    if (h->h_ctl->err) return (blest_status)h->h_ctl->err;
    h->last_levels = h->h_ctl->nlevels;
    return BLEST_OK;
}

// Switching probe (§7.1): three BFSs from fixed sources, with and without
// bottom-up switching; switching stays on only if it was faster overall.
static blest_status probe_switching(blest_graph *h) {
    std::vector<int> deg((size_t)h->n);
    if (cudaMemcpy(deg.data(), h->g.deg, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return BLEST_ERR_CUDA;
    std::vector<int> src;
    unsigned long long x = 0x9E3779B97F4A7C15ull;
    for (int tries = 0; tries < 1000000 && (int)src.size() < 3; ++tries) {
        x ^= x >> 12; x ^= x << 25; x ^= x >> 27;  // xorshift64*
        const long long v = (long long)((x * 0x2545F4914F6CDD1Dull) % (unsigned long long)h->n);
        if (deg[(size_t)v] > 0) src.push_back((int)v);
    }
    if (src.empty()) { h->switching = 0; return BLEST_OK; }
    int *out = nullptr;
    if (cudaMalloc(&out, (size_t)h->n * sizeof(int)) != cudaSuccess) return BLEST_ERR_OOM;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float t[2] = {0.f, 0.f};
    const int saved_async = h->async;
    h->async = 0;
    blest_status st = BLEST_OK;
    for (int rep = 0; rep < 2 && st == BLEST_OK; ++rep) {      // rep 0 warms up
        for (int sw = 0; sw < 2 && st == BLEST_OK; ++sw) {
            h->switching = sw;
            for (int s : src) {
                cudaEventRecord(a, h->stream);
                st = bfs_run(h, s, out);
                if (st != BLEST_OK) break;
                cudaEventRecord(b, h->stream);
                st = finish_call(h, true);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep == 1) t[sw] += ms;
            }
        }
    }
    h->async = saved_async;
    h->switching = (st == BLEST_OK && t[1] < t[0]) ? 1 : 0;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    return st;
}

extern "C" blest_status blest_build(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                    const blest_build_opts *opts, blest_handle *out) {
    if (!out) return BLEST_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n >= ((int64_t)1 << 31) - 64 || !row_ptr || !col_idx) return BLEST_ERR_INVALID;
    blest_build_opts o;
    blest_default_opts(&o);
    if (opts) o = *opts;
    if (o.sigma == 0) o.sigma = 8;
    if (o.sigma != 8 && o.sigma != 16 && o.sigma != 32) return BLEST_ERR_INVALID;
    if (o.tau == 0) o.tau = 32 * (32 / o.sigma);
    if (!bvss_layout_ok(o.sigma, o.tau)) return BLEST_ERR_INVALID;
    if (o.engine_tc && !(o.sigma == 8 && o.tau == 128)) return BLEST_ERR_UNSUPPORTED;
    if (o.block_threads == 0) o.block_threads = 512;
    if (o.block_threads != 256 && o.block_threads != 512 && o.block_threads != 1024) return BLEST_ERR_INVALID;
    if (o.vss_batch == 0) o.vss_batch = 2;
    if (o.vss_batch != 1 && o.vss_batch != 2 && o.vss_batch != 4) return BLEST_ERR_INVALID;
    if (o.timeout_ms <= 0) o.timeout_ms = 5000;
    if (o.reorder < 0 || o.reorder > BLEST_REORDER_AUTO) return BLEST_ERR_INVALID;
    if (o.jaccard_window <= 0) o.jaccard_window = 65536;
    if (o.jaccard_window % o.sigma) return BLEST_ERR_INVALID;

    blest_graph *h = new blest_graph();
    h->n = n;
    h->sigma = o.sigma;
    h->tau = o.tau;
    h->directed = o.directed ? 1 : 0;
    h->engine_tc = o.engine_tc ? 1 : 0;
    h->eta = o.eta > 0 ? o.eta : 10.f;
    h->udiv_threshold = o.udiv_threshold;
    h->timeout_ms = o.timeout_ms;
    h->block = o.block_threads;
    h->vss_batch = o.vss_batch;
    h->fixed_mode = h->engine_tc ? BLEST_MODE_PUSH_EAGER_TC : BLEST_MODE_PUSH_EAGER_CC;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_ctl, sizeof(Ctl));
    if (e != cudaSuccess) {
        blest_internal_record_cuda_error(e, "blest_build setup", __FILE__, __LINE__);
        cudaGetLastError();
        free_all(h);
        delete h;
        return BLEST_ERR_CUDA;
    }
    h->stream = h->own_stream;
    blest_status st = build_graph(h, row_ptr, col_idx, &o);
    if (st == BLEST_OK) st = bfs_prepare(h);
    if (st == BLEST_OK) {
        h->lazy = h->udiv > h->udiv_threshold ? 1 : 0;
        h->switching = 0;
        if (h->lazy && o.probe_switch) st = probe_switching(h);
        else if (h->lazy) h->switching = 1;
    }
    if (st != BLEST_OK) {
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return BLEST_OK;
}

static int32_t *stage_buffer(blest_graph *h, size_t count, blest_status *st) {
    static_assert(sizeof(int32_t) == sizeof(int), "int32");
    if (!h->w.stage || h->w.stage_count < count) {
        void *p = nullptr;
        *st = dev_alloc(h, &p, count * sizeof(int32_t) + 16);
        if (*st != BLEST_OK) return nullptr;
        h->w.stage = (int32_t *)p;
        h->w.stage_count = count;
    }
    *st = BLEST_OK;
    return h->w.stage;
}

extern "C" blest_status blest_bfs(blest_handle h, int32_t source, int32_t *levels) {
    if (!h || !levels || h->many) return BLEST_ERR_INVALID;
    if (source < 0 || (int64_t)source >= h->n) return BLEST_ERR_INVALID;
    const bool dev = is_device_ptr(levels);
    blest_status st = BLEST_OK;
    int32_t *target = dev ? levels : stage_buffer(h, (size_t)h->n, &st);
    if (st != BLEST_OK) return st;
    st = bfs_run(h, source, target);
    if (st != BLEST_OK) return st;
    if (!dev) {
        cudaError_t e = cudaMemcpyAsync(levels, target, (size_t)h->n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                        h->stream);
        if (e != cudaSuccess) return BLEST_ERR_CUDA;
    }
    return finish_call(h, !dev);
}

extern "C" blest_status blest_set_policy(blest_handle h, int32_t policy, int32_t fixed_mode) {
    if (!h || policy < 0 || policy > BLEST_POLICY_SCHEDULE) return BLEST_ERR_INVALID;
    if (policy == BLEST_POLICY_FIXED && (fixed_mode < 0 || fixed_mode >= BLEST_NUM_MODES)) return BLEST_ERR_INVALID;
    if (policy == BLEST_POLICY_LEARNED && !h->d_mlp) return BLEST_ERR_INVALID;
    h->policy = policy;
    if (policy == BLEST_POLICY_FIXED) h->fixed_mode = fixed_mode;
    return BLEST_OK;
}

extern "C" blest_status blest_set_engine(blest_handle h, int32_t tc) {
    if (!h || tc < 0 || tc > 2) return BLEST_ERR_INVALID;
    if (tc && !(h->sigma == 8 && h->tau == 128)) return BLEST_ERR_UNSUPPORTED;
    h->engine_tc = tc;
    return BLEST_OK;
}

extern "C" blest_status blest_set_launch(blest_handle h, int32_t block_threads, int32_t vss_batch) {
    if (!h || h->many) return BLEST_ERR_INVALID;
    if (block_threads != 256 && block_threads != 512 && block_threads != 1024) return BLEST_ERR_INVALID;
    if (vss_batch != 1 && vss_batch != 2 && vss_batch != 4) return BLEST_ERR_INVALID;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    const int g = bfs_grid_for(h, block_threads, nullptr);
    if (g <= 0) return BLEST_ERR_CUDA;
    h->block = block_threads;
    h->grid = g;
    h->vss_batch = vss_batch;
    return BLEST_OK;
}

extern "C" blest_status blest_set_queue_deferral(blest_handle h, int32_t mode) {
    if (!h || h->many || mode < -1 || mode > 1) return BLEST_ERR_INVALID;
    h->defer_queue = mode;
    return BLEST_OK;
}

extern "C" blest_status blest_set_switching(blest_handle h, int32_t on) {
    if (!h || h->many || (on != 0 && on != 1)) return BLEST_ERR_INVALID;
    h->switching = on;
    return BLEST_OK;
}

extern "C" blest_status blest_set_schedule(blest_handle h, const int32_t *modes, int32_t len) {
    if (!h || !modes || len <= 0 || len > (1 << 20)) return BLEST_ERR_INVALID;
    std::vector<int32_t> m((size_t)len);
    if (cudaMemcpy(m.data(), modes, (size_t)len * sizeof(int32_t), cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    for (int32_t x : m)
        if (x < 0 || x >= BLEST_NUM_MODES) return BLEST_ERR_INVALID;
    if (len > h->sched_len) {
        blest_status st = dev_alloc_t(h, &h->d_schedule, (size_t)len);
        if (st != BLEST_OK) return st;
    }
    if (cudaMemcpy(h->d_schedule, m.data(), (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return BLEST_ERR_CUDA;
    h->sched_len = len;
    return BLEST_OK;
}

extern "C" blest_status blest_load_model(blest_handle h, const float *weights, int32_t nweights) {
    if (!h || !weights || nweights != MLP_NW) return BLEST_ERR_INVALID;
    if (!h->d_mlp) {
        blest_status st = dev_alloc_t(h, &h->d_mlp, (size_t)MLP_NW);
        if (st != BLEST_OK) return st;
    }
    if (cudaMemcpyAsync(h->d_mlp, weights, (size_t)MLP_NW * sizeof(float), cudaMemcpyDefault, h->stream) !=
        cudaSuccess)
        return BLEST_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    h->mlp_len = MLP_NW;
    return BLEST_OK;
}

extern "C" blest_status blest_last_timings(blest_handle h, blest_level_log *buf, int64_t cap, int64_t *len) {
    if (!h || !len) return BLEST_ERR_INVALID;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    int64_t nl = h->last_levels;
    if (nl > h->w.log_cap) nl = h->w.log_cap;
    *len = nl;
    if (buf && cap > 0) {
        const int64_t k = nl < cap ? nl : cap;
        if (k > 0 && cudaMemcpy(buf, h->w.log, (size_t)k * sizeof(blest_level_log), cudaMemcpyDefault) != cudaSuccess)
            return BLEST_ERR_CUDA;
    }
    return BLEST_OK;
}

extern "C" blest_status blest_get_info(blest_handle h, blest_info *info) {
    if (!h || !info) return BLEST_ERR_INVALID;
    memset(info, 0, sizeof *info);
    info->n = h->n;
    info->nnz = h->nnz;
    info->num_slice_sets = h->Ns;
    info->num_vss = h->Nv;
    info->num_slices = h->num_slices;
    info->update_divergence = h->udiv;
    info->lazy = h->lazy;
    info->switching = h->switching;
    info->reorder = h->reorder;
    info->sigma = h->sigma;
    info->tau = h->tau;
    info->vss_batch = h->vss_batch;
    info->grid_blocks = h->grid;
    info->block_threads = h->block;
    info->build_ms = h->build_ms;
    info->device_bytes = h->device_bytes;
    info->policy = h->policy;
    info->engine_tc = h->engine_tc;
    info->model_loaded = h->d_mlp != nullptr;
    return BLEST_OK;
}

extern "C" blest_status blest_get_bvss(blest_handle h, int32_t *row_ids, uint32_t *masks, int32_t *real_ptrs,
                                       int32_t *v2r) {
    if (!h || h->many) return BLEST_ERR_INVALID;
    cudaStreamSynchronize(h->stream);
    const size_t nv = (size_t)h->Nv;
    const size_t tau = (size_t)h->tau, words = tau / (size_t)(32 / h->sigma);
    if (row_ids && nv && cudaMemcpy(row_ids, h->g.rowIds, nv * tau * 4, cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (masks && nv && cudaMemcpy(masks, h->g.masks, nv * words * 4, cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (real_ptrs && cudaMemcpy(real_ptrs, h->g.realPtrs, ((size_t)h->Ns + 1) * 4, cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (v2r && nv && cudaMemcpy(v2r, h->g.v2r, nv * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    return BLEST_OK;
}

extern "C" blest_status blest_get_perm(blest_handle h, int32_t *new_of_old) {
    if (!h || !new_of_old || h->many) return BLEST_ERR_INVALID;
    cudaStreamSynchronize(h->stream);
    if (!h->g.new_of_old) {
        std::vector<int32_t> id((size_t)h->n);
        for (int64_t i = 0; i < h->n; ++i) id[(size_t)i] = (int32_t)i;
        if (cudaMemcpy(new_of_old, id.data(), (size_t)h->n * 4, cudaMemcpyDefault) != cudaSuccess)
            return BLEST_ERR_CUDA;
        return BLEST_OK;
    }
    if (cudaMemcpy(new_of_old, h->g.new_of_old, (size_t)h->n * 4, cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    return BLEST_OK;
}

extern "C" blest_status blest_set_stream(blest_handle h, void *stream, int32_t async) {
    if (!h) return BLEST_ERR_INVALID;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    h->async = async ? 1 : 0;
    return BLEST_OK;
}

extern "C" blest_status blest_sync(blest_handle h) {
    if (!h) return BLEST_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return BLEST_ERR_CUDA;
    if (h->h_ctl->err) {
        blest_status s = (blest_status)h->h_ctl->err;
        return s;
    }
    h->last_levels = h->h_ctl->nlevels;
    return BLEST_OK;
}

extern "C" void blest_destroy(blest_handle h) {
    if (!h) return;
    free_all(h);
    delete h;
}

extern "C" const char *blest_status_string(blest_status s) {
    switch (s) {
        case BLEST_OK: return "ok";
        case BLEST_ERR_INVALID: return "invalid argument";
        case BLEST_ERR_OOM: return "out of memory";
        case BLEST_ERR_CUDA: return "CUDA error";
        case BLEST_ERR_TIMEOUT: return "device wait timed out";
        case BLEST_ERR_UNSUPPORTED: return "unsupported";
        case BLEST_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

// ------------------------------------------------------- barrier self-test
namespace {
__global__ void k_barrier_selftest(Ctl *ctl, unsigned long long budget_ns) {
    if (blockIdx.x != 0) return;  // block 1 never arrives
    unsigned epoch = 0;
    grid_barrier(ctl, epoch, budget_ns);
}
}  // namespace

extern "C" blest_status blest_selftest_barrier_timeout(int32_t timeout_ms) {
    if (timeout_ms <= 0 || timeout_ms > 10000) return BLEST_ERR_INVALID;
    Ctl *d = nullptr;
    if (cudaMalloc(&d, sizeof(Ctl)) != cudaSuccess) return BLEST_ERR_CUDA;
    cudaMemset(d, 0, sizeof(Ctl));
    k_barrier_selftest<<<2, 32>>>(d, (unsigned long long)timeout_ms * 1000000ull);
    cudaError_t e = cudaDeviceSynchronize();
    Ctl hc;
    memset(&hc, 0, sizeof hc);
    if (e == cudaSuccess) e = cudaMemcpy(&hc, d, sizeof(Ctl), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return BLEST_ERR_CUDA;
    return (blest_status)hc.err;
}
