// Host-side state of a blest handle (shared by the translation units of the
// library; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/blest.h"
#include "common.cuh"

struct DevGraph {
    // BVSS (§3.1): rowIds int32[N_v*tau] (slice k of VSS v at v*tau + k;
    // lane word l owns slots l*theta .. l*theta + theta - 1, one vector load),
    // masks u32[N_v*tau/theta] (slice c of a word in bits [c*sigma, (c+1)*sigma)),
    // theta = 32/sigma
    int *rowIds = nullptr;
    unsigned *masks = nullptr;
    int *realPtrs = nullptr;   // N_s + 1
    int *v2r = nullptr;        // N_v
    // in-neighbour CSR of the reordered graph (bottom-up, Algorithm 4)
    long long *rp = nullptr;   // n + 1
    int *col = nullptr;
    int *deg = nullptr;        // out-degree in the reordered id space (features, TEPS)
    unsigned *nz = nullptr;    // bit u set iff u has an in-neighbour (bottom-up skips the rest)
    int4 *head = nullptr;      // first four in-neighbours of each vertex (bottom-up first probe)
    // permutation (nullptr when no reordering): new_of_old, old_of_new
    int *new_of_old = nullptr;
    int *old_of_new = nullptr;
};

struct BfsWork {
    int *L = nullptr;                 // n (reordered ids)
    unsigned *Vc = nullptr, *Vn = nullptr;
    unsigned *F[3] = {nullptr, nullptr, nullptr};
    int2 *Q[3] = {nullptr, nullptr, nullptr};   // {VSS id, slice set}
    int *SQ[3] = {nullptr, nullptr, nullptr};
    Ctl *ctl = nullptr;
    blest_level_log *log = nullptr;
    int log_cap = 0;
    int *out_tmp = nullptr;           // n, levels in reordered ids (when reordered)
    int32_t *stage = nullptr;         // device staging for host outputs
    size_t stage_count = 0;
};

struct MsbfsWork;  // defined in msbfs.cu
struct ManyGraphs; // defined in many.cu

struct blest_graph {
    int64_t n = 0, nnz = 0;
    int64_t Ns = 0, Nv = 0, num_slices = 0;
    int sigma = 8;
    int tau = 128;                    // slices per VSS
    int directed = 0;
    int reorder = 0;
    double udiv = 0.0;
    int lazy = 0, switching = 0;
    int engine_tc = 1;
    int ms_engine = 0;                // multi-source stage 1: 0 CUDA cores, 1 tcgen05 (tau = 128)
    int ms_remap = 1, ms_track = 1;   // multi-source variant: getVI order, activeSets / dirtySets
    int defer_queue = -1;             // deferred VSS queues: -1 on graphs with bottom-up switching, 0 off, 1 on
    int ms_dir = 0;                   // multi-source stage 1: 0 push, 1 pull on dense levels, 2 pull
    int ms_out = 1;                   // multi-source levels: 1 staged as bytes, then transposed; 0 direct
    int vss_batch = 2;
    float eta = 10.f;
    double udiv_threshold = 25000.0;
    int timeout_ms = 5000;
    double build_ms = 0.0;
    int64_t device_bytes = 0;

    DevGraph g;
    BfsWork w;

    // launch geometry of the persistent kernels
    int block = 512;
    int grid = 0;
    int num_sms = 0;
    int device = 0;

    // policy
    int policy = BLEST_POLICY_HEURISTIC;
    int fixed_mode = BLEST_MODE_PUSH_EAGER_TC;
    int *d_schedule = nullptr;
    int sched_len = 0;
    float *d_mlp = nullptr;
    int mlp_len = 0;

    // streams and status
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int async = 0;
    Ctl *h_ctl = nullptr;             // pinned copy of the control block
    int last_levels = 0;

    MsbfsWork *ms = nullptr;
    ManyGraphs *many = nullptr;

    std::vector<void *> allocations;  // every device allocation, freed at destroy
};

// allocation helper: records the pointer in the handle
blest_status dev_alloc(blest_graph *h, void **p, size_t bytes);
template <typename T>
static inline blest_status dev_alloc_t(blest_graph *h, T **p, size_t count) {
    return dev_alloc(h, (void **)p, count * sizeof(T) + 16);
}

// is this pointer device-accessible memory?
bool is_device_ptr(const void *p);

// build helpers (build.cu)
blest_status build_graph(blest_graph *h, const int64_t *row_ptr, const int32_t *col_idx,
                         const blest_build_opts *o);

// BFS (bfs.cu)
blest_status bfs_prepare(blest_graph *h);
blest_status bfs_run(blest_graph *h, int32_t source, int32_t *levels_dev_out);
int bfs_grid_for(const blest_graph *h, int block, int *num_sms);

// the (sigma, tau) pairs the kernels are built for: (8, 32), (8, 128), (16, 64), (32, 32)
static inline bool bvss_layout_ok(int sigma, int tau) {
    return (sigma == 8 && (tau == 32 || tau == 128)) || (sigma == 16 && tau == 64) || (sigma == 32 && tau == 32);
}
