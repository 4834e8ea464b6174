/*
 * blest.h -- C ABI of the GB300 (sm_103a) BVSS breadth-first-search library.
 *
 * The library implements the data-parallel path of "Graph Traversal on
 * Tensor Cores: A BFS Framework for Modern GPUs" (Elbek & Kaya): BFS as a
 * binary sparse-matrix x sparse-frontier product (§2, Eq. 1-2) over the
 * Binarized Virtual Slice Set layout (§3.1), with eager (Algorithm 2) and
 * lazy (Algorithm 3) vertex updates, bottom-up levels (Algorithm 4) behind a
 * per-level switch (Eq. 5), multi-source BFS (§6.1, Algorithm 5) and exact
 * closeness centrality (§6.2, Eq. 6-7).
 *
 * Conventions shared by every entry point
 *  - Graphs are CSR: row_ptr (int64, n+1 entries, row_ptr[0] = 0,
 *    non-decreasing) and col_idx (int32, row_ptr[n] entries, each in [0, n)).
 *    Row v lists the out-neighbours of v.  An undirected graph is given as a
 *    symmetric CSR.  Rows need not be sorted; duplicate arcs and self loops
 *    are ignored (they change no BFS level).
 *  - Input arrays are caller-owned and may be host or device memory; they are
 *    copied during the call and not retained.
 *  - Output arrays are caller-allocated and may be host or device memory
 *    (detected with cudaPointerGetAttributes).  Vertex ids in outputs are
 *    always the caller's original ids: any reordering done by blest_build is
 *    undone on the device.
 *  - Levels are int32 hop distances from the source; unreached = -1.
 *  - Every call is ordered on the handle's CUDA stream (blest_set_stream).
 *    By default a call returns after its work is complete and reports any
 *    device-side error (for example a grid-barrier timeout).  In asynchronous
 *    mode a call whose outputs are all device memory returns after enqueueing
 *    and blest_sync() reports the device status.
 *  - A handle is not thread-safe: calls on one handle must be serialised.
 *    Different handles may be used concurrently.
 *  - On BLEST_ERR_INVALID the outputs are untouched.
 */
#ifndef BLEST_H
#define BLEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct blest_graph *blest_handle;

typedef enum {
    BLEST_OK = 0,
    BLEST_ERR_INVALID = 1,     /* bad argument, malformed CSR, source out of range */
    BLEST_ERR_OOM = 2,         /* device or pinned-host allocation failed */
    BLEST_ERR_CUDA = 3,        /* a CUDA runtime call failed (no GPU, launch failure) */
    BLEST_ERR_TIMEOUT = 4,     /* a device-side wait exceeded its time budget */
    BLEST_ERR_UNSUPPORTED = 5, /* valid request this build or graph does not support */
    BLEST_ERR_INTERNAL = 6     /* a device-side consistency check failed */
} blest_status;

/* Vertex reordering applied by blest_build (§4).  On a directed graph the
 * ordering is computed on its symmetrised pattern G + G^T (RCM is defined for
 * symmetric patterns); the permutation changes speed, never levels. */
enum {
    BLEST_REORDER_NONE = 0,
    BLEST_REORDER_RCM = 1,      /* reverse Cuthill-McKee (§4.2) */
    BLEST_REORDER_JACCARD = 2,  /* JaccardWithWindows (§4.1, Algorithm 1) */
    BLEST_REORDER_AUTO = 3      /* Jaccard if scale-free-like (§4.2 footnote), else RCM */
};

/* Per-level kernel choices. */
enum {
    BLEST_MODE_PUSH_EAGER_CC = 0,  /* Algorithm 2, CUDA-core AND + byte test */
    BLEST_MODE_PUSH_EAGER_TC = 1,  /* Algorithm 2, m8n8k128 b1 AND.POPC (Fig. 3 layout) */
    BLEST_MODE_PUSH_LAZY_CC = 2,   /* Algorithm 3 stage 1 on CUDA cores + stage 2 */
    BLEST_MODE_PUSH_LAZY_TC = 3,   /* Algorithm 3 stage 1 on tensor cores + stage 2 */
    BLEST_MODE_BOTTOM_UP = 4,      /* Algorithm 4 + stage 2 */
    BLEST_NUM_MODES = 5
};

/* How the per-level mode is chosen. */
enum {
    BLEST_POLICY_HEURISTIC = 0, /* §5.3/§7.1: eager vs lazy by U_div, bottom-up by Eq. 5 */
    BLEST_POLICY_LEARNED = 1,   /* MLP over per-level features (weights via blest_load_model) */
    BLEST_POLICY_FIXED = 2,     /* one mode for every level (fixed_mode) */
    BLEST_POLICY_SCHEDULE = 3   /* per-level modes from blest_set_schedule (testing) */
};

typedef struct blest_build_opts {
    int32_t reorder;         /* BLEST_REORDER_*; default NONE */
    int32_t sigma;           /* slice width: 8 (default), 16 or 32 (§3.1) */
    int32_t directed;        /* 0: CSR is symmetric (undirected); 1: directed */
    int32_t jaccard_window;  /* W of Algorithm 1; default 65536, multiple of sigma */
    int32_t probe_switch;    /* 1 (default): the 3-source switching probe of §7.1 runs at build */
    int32_t engine_tc;       /* top-down hit test: 1 = b1 MMA (Fig. 3 layout), 0 (default) = CUDA
                                cores (measured faster on GB300) */
    float eta;               /* Eq. 5 constant; default 10 */
    double udiv_threshold;   /* lazy if U_div > threshold (§7.1); default 25000 */
    int32_t timeout_ms;      /* budget of each device-side wait; default 5000 */
    int32_t block_threads;   /* CTA size of the persistent kernels: 256, 512 or 1024; 0 = 512 */
    int32_t vss_batch;       /* VSSs a warp keeps in flight in top-down levels: 1, 2, 4; 0 = 2 */
    int32_t tau;             /* slices per VSS.  0 = 32 * (32 / sigma), the warp-wide VSS of §3.1
                                (sigma 8: 128, 16: 64, 32: 32).  sigma = 8 also takes 32: a VSS
                                spans 8 lanes and a warp works on four at once (for graphs whose
                                slice sets hold few slices, e.g. road-like grids) */
} blest_build_opts;

/* Build-time facts about a handle. */
typedef struct blest_info {
    int64_t n, nnz;          /* vertices, distinct non-loop arcs */
    int64_t num_slice_sets;  /* N_s */
    int64_t num_vss;         /* N_v */
    int64_t num_slices;
    double update_divergence;/* U_div (§4.2) */
    int32_t lazy;            /* 1 if the heuristic policy uses Algorithm 3 */
    int32_t switching;       /* 1 if bottom-up switching is enabled */
    int32_t reorder;         /* the reordering actually applied */
    int32_t sigma;
    int32_t grid_blocks;     /* persistent-kernel grid */
    int32_t block_threads;
    double build_ms;         /* device time of the build */
    int64_t device_bytes;    /* device memory held by the handle */
    int32_t tau;             /* slices per VSS */
    int32_t vss_batch;       /* VSS passes a warp keeps in flight (launch setting) */
    int32_t policy;          /* blest_policy in force */
    int32_t engine_tc;       /* 1: the rule and fixed policies run the b1-MMA hit test of Fig. 3 */
    int32_t model_loaded;    /* 1 once MLP weights are loaded; without them LEARNED falls back to the rule */
} blest_info;

/* One record per BFS level of the last single-source BFS. */
typedef struct blest_level_log {
    int32_t level;           /* level being computed (1 = neighbours of the source) */
    int32_t mode;            /* BLEST_MODE_* that ran */
    int64_t frontier;        /* |X_{level-1}|: vertices in the input frontier */
    int64_t frontier_edges;  /* out-arcs of those vertices */
    int64_t unvisited;       /* vertices not visited before this level */
    int64_t queue;           /* |Q_curr|: VSSs scheduled */
    int64_t t_ns;            /* device time of the level (globaltimer) */
    int64_t scanned_vertices;/* bottom-up levels: unvisited vertices probed */
    int64_t scanned_arcs;    /* bottom-up levels: in-neighbour ids read beyond each row's first four */
    int64_t slots;           /* BVSS slots scheduled: tau * queue (the active-slice input of the
                                learned policy) */
    int64_t t_stage1_ns;     /* device time of stage 1 alone (lazy and bottom-up levels; equals t_ns
                                for eager levels) */
    int64_t vss_batch;       /* VSS passes a warp kept in flight (top-down levels) */
} blest_level_log;

/* Fill *opts with the defaults documented above. */
void blest_default_opts(blest_build_opts *opts);

/* Build a handle from a CSR graph (§3.1 BVSS construction, §4 reordering).
 * n >= 1.  opts may be NULL (defaults).  The handle owns all device memory
 * and must be released with blest_destroy.  Returns INVALID for a malformed
 * CSR or a sigma / tau pair other than (8, 32), (8, 128), (16, 64),
 * (32, 32); UNSUPPORTED for n >= 2^31, for engine_tc = 1 with a layout other
 * than sigma = 8, tau = 128 (the Fig. 3 fragment layout), or when the BVSS
 * would need 2^31 or more lane words (N_v * tau / theta). */
blest_status blest_build(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                         const blest_build_opts *opts, blest_handle *out);

/* Single-source BFS (Algorithms 2-4 under the handle's policy).
 * levels: n int32 values, indexed by original vertex id. */
blest_status blest_bfs(blest_handle h, int32_t source, int32_t *levels);

/* Multi-source BFS (§6.1, Algorithm 5): k sources (1 <= k <= 1024,
 * duplicates allowed) as bit lanes.  levels: k*n int32, levels[c*n + v] is
 * the distance from sources[c] to v.  Needs sigma = 8 (getVI of §6.1 groups
 * the eight vertices of a slice set); UNSUPPORTED otherwise, and so are the
 * closeness calls below. */
blest_status blest_msbfs(blest_handle h, const int32_t *sources, int32_t k, int32_t *levels);

/* Stage-1 engine of the multi-source kernel (and of closeness): 0 (default)
 * = CUDA cores (the OR of the frontier elements each slice mask selects, 32
 * lanes per 32-bit operation); 1 = the fifth-generation tensor cores:
 * Eq. 2 for a 128-lane tile of the frontier and 64 slots of a VSS as one
 * tcgen05 kind::f16 MMA with 0/1 bf16 operands (K = the slice set's 8
 * columns, zero-padded to 16) and fp32 sums in tensor memory, a lane
 * reaching a slot's row iff its sum is nonzero.  Levels are identical.
 * The tensor-core engine needs sigma = 8, tau = 128 (UNSUPPORTED
 * otherwise). */
blest_status blest_set_msbfs_engine(blest_handle h, int32_t tc);

/* Direction of the multi-source stage 1.  0 = push (Algorithm 5: each
 * active VSS ORs its slots' hit words into V_next with atomics; the
 * default); 2 = pull: every vertex with an unvisited lane ORs the frontier
 * elements of its in-neighbours (stopping once all its unvisited lanes are
 * reached) and writes its own V_next word, no atomics; 1 = pull on levels
 * whose queue holds more than an eighth of the VSSs, push on the others.
 * Pulling reaches exactly the lanes pushing does (Eq. 2 read by row);
 * levels are identical.  Pull levels run on CUDA cores whatever the
 * stage-1 engine.  Measured on GB300 (RMAT 22, 1024 lanes): push 127 ms,
 * 1: 158 ms, 2: 192 ms -- each pulled in-neighbour is a dependent
 * 128-byte read, slower than the atomics it replaces. */
blest_status blest_set_msbfs_direction(blest_handle h, int32_t mode);

/* Variant of the multi-source kernel (for the ablation of §7.1): reindex =
 * 1 stores vertex u's kappa-bit element at getVI(u) (§6.1), 0 at u;
 * tracking = 1 visits only the active slice sets' VSSs in stage 1 and the
 * dirty slice sets in stage 2 (activeSets / dirtySets of Algorithm 5), 0
 * every VSS and every slice set at every level.  Default (1, 1) is
 * Algorithm 5 in full; (0, 0) and (1, 0) are the ablation's (A) and (AB).
 * Levels are identical.  The tensor-core engine runs only (1, 1). */
blest_status blest_set_msbfs_variant(blest_handle h, int32_t reindex, int32_t tracking);

/* How blest_msbfs writes its k x n source-major levels (not a step of the
 * paper, which gives no output layout).  staged = 1 (default): stage 2 keeps
 * one byte per (vertex, lane) in vertex-major rows of kappa bytes (levels
 * 0..253; deeper levels go straight to the output), and after the last level
 * the kernel transposes the rows into the output with coalesced stores; the
 * handle allocates the rows (ceil(n/8) * 8 * kappa bytes) at the first
 * blest_msbfs.  staged = 0: one int32 store per reached (vertex, lane) in
 * stage 2, after a -1 fill of the output.  Levels are identical. */
blest_status blest_set_msbfs_output(blest_handle h, int32_t staged);

/* Exact closeness centrality by all-source BFS in 1024-lane batches (§6.2).
 * far: n int64 distance sums (Eq. 6); cc: n doubles, cc[u] = (reach[u]-1) /
 * far[u] (Eq. 7 with component-size normalisation; 0 when far[u] = 0), may be
 * NULL; reach: n int64 component sizes, may be NULL.  Undirected graphs only
 * (UNSUPPORTED otherwise).  Each batch is one replay of a CUDA graph (source
 * ids from a device cursor, the persistent multi-source kernel, the cursor
 * advance) captured on the handle's stream at the first call, so that stream
 * must allow capture (the handle's own stream does; cudaStreamLegacy does
 * not). */
blest_status blest_closeness(blest_handle h, int64_t *far, double *cc, int64_t *reach);

/* Partial closeness: distance sums from the sources with original ids
 * [first, first + count) only, written (not accumulated) to far and reach
 * (n int64 each, reach may be NULL).  Sums over disjoint ranges add up to
 * the full result; this is how an all-source run is split across calls,
 * processes or GPUs.  Undirected graphs only. */
blest_status blest_closeness_range(blest_handle h, int64_t first, int64_t count, int64_t *far,
                                   int64_t *reach);

/* Work counters of the last blest_msbfs, blest_closeness or
 * blest_closeness_range call on the handle, summed over its launches (one
 * per batch of up to kappa sources): the terms of the multi-source byte
 * model (stage 1 loads each processed VSS and its slice set's frontier
 * elements and ORs each nonzero hit word into V_next; stage 2 reads and
 * writes the kappa-bit elements of the eight vertices of each dirty set). */
typedef struct blest_msbfs_counters {
    int64_t kappa;        /* lanes per batch: 64, 256 or 1024 */
    int64_t launches;     /* persistent-kernel launches */
    int64_t levels;       /* levels, summed over the launches */
    int64_t vss;          /* VSSs processed in stage 1 */
    int64_t hit_words;    /* nonzero 32-lane words OR-ed into V_next */
    int64_t dirty_sets;   /* slice sets finalised in stage 2 */
    int64_t pull_levels;  /* levels whose stage 1 pulled (blest_set_msbfs_direction) */
    int64_t pull_arcs;    /* in-neighbour elements read by pulling vertices */
} blest_msbfs_counters;

blest_status blest_msbfs_stats(blest_handle h, blest_msbfs_counters *out);

/* Many small graphs in one handle: graph i has vertices [vtx_off[i],
 * vtx_off[i+1]) (local ids from 0) and arcs [edge_off[i], edge_off[i+1]);
 * its local row pointer is row_ptr[vtx_off[i] + i .. vtx_off[i+1] + i]
 * (offsets relative to edge_off[i]).  Undirected graphs only; the BVSS is
 * the default sigma = 8, tau = 128 one (other sigma / tau: UNSUPPORTED). */
blest_status blest_build_many(int32_t g, const int64_t *vtx_off, const int64_t *edge_off,
                              const int64_t *row_ptr, const int32_t *col_idx_local,
                              const blest_build_opts *opts, blest_handle *out);

/* One BFS per graph of a blest_build_many handle, all in one persistent
 * launch.  sources: g local ids; levels: sum of n_i int32, graph i at
 * vtx_off[i]. */
blest_status blest_bfs_many(blest_handle h, const int32_t *sources, int32_t *levels);

/* Choose the per-level policy.  fixed_mode is used by BLEST_POLICY_FIXED. */
blest_status blest_set_policy(blest_handle h, int32_t policy, int32_t fixed_mode);

/* Hit-test engine of the heuristic policy's top-down levels: 1 = b1 MMA
 * (Fig. 3 layout, the paper's: 2 MMAs per 128 slices), 0 = CUDA cores, 2 =
 * b1 MMA with one slice per fragment row (16 MMAs per 128 slices, the
 * layout Fig. 3 improves on; for the ablation).  Tensor-core modes of a
 * fixed policy or schedule use the same layout.  The MMA needs sigma = 8,
 * tau = 128 (UNSUPPORTED otherwise); on other layouts a fixed policy or
 * schedule that names a tensor-core mode runs its CUDA-core twin, and the
 * level log records the mode that ran. */
blest_status blest_set_engine(blest_handle h, int32_t tc);

/* Launch shape of the single-source kernel: block_threads in {256, 512,
 * 1024}, vss_batch in {1, 2, 4} (VSSs a warp keeps in flight in top-down
 * levels).  The grid is resized to the SMs' resident capacity. */
blest_status blest_set_launch(blest_handle h, int32_t block_threads, int32_t vss_batch);

/* Eq. 5 bottom-up switching of the heuristic policy on (1) or off (0).  The
 * build decides it (§7.1: by the three-source probe for graphs that use
 * lazy updates, off otherwise); this overrides that decision. */
blest_status blest_set_switching(blest_handle h, int32_t on);

/* Deferred VSS queues (not a step of the paper): a lazy (Algorithm 3) or
 * bottom-up (Algorithm 4) level counts the VSS queue of the next level and
 * writes only its slice-set list; a top-down level that follows writes the
 * queue from that list first (one pass and a grid barrier), while a
 * bottom-up level, which reads only the frontier bits, skips it.  mode = 1
 * on, 0 off, -1 (the default) on exactly when bottom-up switching is on.
 * Levels are identical. */
blest_status blest_set_queue_deferral(blest_handle h, int32_t mode);

/* Per-level modes for BLEST_POLICY_SCHEDULE: level l (1-based) runs
 * modes[(l-1) % len].  Copied. */
blest_status blest_set_schedule(blest_handle h, const int32_t *modes, int32_t len);

/* Load MLP weights for BLEST_POLICY_LEARNED (layout in blest_mlp_*). */
blest_status blest_load_model(blest_handle h, const float *weights, int32_t nweights);

/* Copy the per-level log of the last blest_bfs into buf (cap records);
 * *len receives the number of levels. */
blest_status blest_last_timings(blest_handle h, blest_level_log *buf, int64_t cap, int64_t *len);

/* Build facts. */
blest_status blest_get_info(blest_handle h, blest_info *info);

/* Copy the device BVSS arrays (§3.1) to caller buffers (host or device):
 * rowIds N_v*tau int32 (slice k of VSS v at v*tau + k), masks N_v*tau/theta
 * uint32 (theta = 32/sigma slices per word, slice c of a word in bits
 * [c*sigma, (c+1)*sigma)), realPtrs N_s+1 int32, virtualToReal N_v int32.
 * Any pointer may be NULL.  Ids are in the reordered space (see
 * blest_get_perm). */
blest_status blest_get_bvss(blest_handle h, int32_t *row_ids, uint32_t *masks, int32_t *real_ptrs,
                            int32_t *virtual_to_real);

/* new_of_old[v] = position of original vertex v after reordering. */
blest_status blest_get_perm(blest_handle h, int32_t *new_of_old);

/* Use a caller CUDA stream (a cudaStream_t, NULL = the handle's own).
 * async = 1: calls with device-only outputs return after enqueueing. */
blest_status blest_set_stream(blest_handle h, void *stream, int32_t async);

/* Wait for the handle's stream and return the device status of the calls
 * since the last sync. */
blest_status blest_sync(blest_handle h);

/* Release the handle and its device memory. */
void blest_destroy(blest_handle h);

const char *blest_status_string(blest_status s);

/* ---- Learned level-mode policy (replaces the hand-set rule of §5.3 / §7.1)
 * A 3-layer MLP (6 -> 32 -> 32 -> 9, tanh, fp32) predicts, from six
 * per-level features, the log device time of each of BLEST_NUM_CHOICES
 * level choices; BLEST_POLICY_LEARNED runs the choice with the smallest
 * prediction.  A choice is a mode and the VSS passes a warp keeps in flight:
 * choices 0-4 are the modes BLEST_MODE_* (lazy ones with one pass), 5 and 6
 * lazy CUDA-core with 2 and 4 passes, 7 and 8 lazy b1-MMA with 2 and 4.
 * Bottom-up is never chosen for a level with more than 16 unvisited
 * vertices per out-arc of its frontier (raw features: log1p(unvisited) >
 * log1p(frontier_edges) + log 16), whatever the prediction.
 * Weights: BLEST_MLP_NW floats, [0,6) feature means, [6,12) feature 1/std,
 * then W1[32][6], b1[32], W2[32][32], b2[32], W3[9][32], b3[9].  All arrays
 * below may be host or device memory and are row-major (one sample per
 * row). */
#define BLEST_NUM_CHOICES 9
#define BLEST_MLP_NW 1589

/* Raw features of level-log records, exactly as the BFS kernel computes
 * them: out[n*6] = log1p of (frontier, frontier_edges, unvisited, slots,
 * level, avg_deg). */
blest_status blest_mlp_features(const blest_level_log *recs, int64_t n, float avg_deg, float *out);

/* Masked mean squared error of the predictions against targets (n*9 log
 * times, mask 1 = observed) and its gradient (BLEST_MLP_NW floats; the
 * normalisation entries get 0). */
blest_status blest_mlp_loss_grad(const float *features, const float *targets, const float *mask, int64_t n,
                                 const float *weights, float *loss, float *grad);

/* Full-batch Adam training on the device, deterministic.  weight_decay adds
 * (weight_decay/2)|w|^2 over the trainable entries to the loss.  weights:
 * in = initial values (normalisation entries included, never updated), out
 * = trained.  loss_out: the data loss before each of the `epochs` steps, may
 * be NULL.  The mask entries weight the squared errors (0 = unobserved). */
blest_status blest_mlp_train(const float *features, const float *targets, const float *mask, int64_t n,
                             int32_t epochs, float lr, float weight_decay, float *weights, float *loss_out);

/* Predictions (n*9, may be NULL) and chosen choices (n, may be NULL) with the
 * in-kernel inference routine. */
blest_status blest_mlp_predict(const float *weights, const float *features, int64_t n, float *pred,
                               int32_t *choice);

/* ---- Allocation-free BFS ------------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot call cudaMalloc: code whose device memory is entirely owned by
 * another allocator (a framework that reserves the whole pool up front) and
 * latency-critical paths where cudaMalloc's implicit device synchronisation
 * is not allowed.  It runs the single-source BFS kernel over a BVSS the
 * caller already holds in device memory (for example copied out of a handle
 * with blest_get_bvss), in a fixed top-down eager mode, and allocates
 * nothing: its scratch (bitvectors, queues, control block, about 5.4 MB)
 * is a static array of the library's device image that every GPU loading
 * the library holds until the process exits.
 *  - Limits: n <= 1,048,576 vertices and num_vss <= 131,072; larger graphs
 *    return BLEST_ERR_UNSUPPORTED.  The BVSS must have the sigma = 8,
 *    tau = 128 layout (the view's sigma and tau fields say so; any other
 *    layout returns BLEST_ERR_UNSUPPORTED).
 *  - Vertex ids are those of the BVSS: for a handle built with reordering,
 *    blest_get_bvss returns the reordered graph, so `source`, `out_degree`
 *    and the levels written are in the reordered numbering (map them with
 *    blest_get_perm: reordered id = new_of_old[original id]).
 *  - The first call on each device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *    That set-up is guarded by a lock, so first calls may come from several
 *    host threads.
 *  - All calls share the scratch array: calls that overlap on the GPU (other
 *    streams or host threads) race.  Each call clears what must start at zero.
 *  - levels must be device memory (n int32).  The call is synchronous: it
 *    launches on `stream` (a cudaStream_t, NULL = the legacy default stream),
 *    waits for that stream and returns the device status. */
typedef struct blest_bvss_view {
    int64_t n;                       /* vertices */
    int64_t num_slice_sets;          /* N_s = ceil(n / 8): sigma = 8, tau = 128 layout only */
    int64_t num_vss;                 /* N_v */
    const int32_t *row_ids;          /* device, N_v*128 (blest_get_bvss layout) */
    const uint32_t *masks;           /* device, N_v*32 */
    const int32_t *real_ptrs;        /* device, N_s + 1 */
    const int32_t *virtual_to_real;  /* device, N_v */
    const int32_t *out_degree;       /* device, n out-degrees (per-level counters) */
    int32_t engine_tc;               /* 1: b1 MMA hit test, 0: CUDA cores */
    int32_t sigma;                   /* slice width of the BVSS: must be 8 */
    int32_t tau;                     /* slices per VSS: must be 128 */
} blest_bvss_view;

blest_status blest_bfs_noalloc(const blest_bvss_view *g, int32_t source, int32_t *levels, void *stream);

/* ---- Scale-free-like test (§4.2 footnote) --------------------------------
 * The test BLEST_REORDER_AUTO applies to choose JaccardWithWindows (scale-
 * free-like) or RCM.  A degree distribution is heavy-tailed when (a) the top
 * 1 % of vertices hold at least 5 % and the top 10 % at least 40 % of the
 * total degree, or (b) a least-squares line through the log-log degree
 * histogram over the degrees k >= 5 has slope -gamma with R^2 >= 0.70 and
 * gamma in [1, 5]; a graph is scale-free-like when its out- or in-degree
 * distribution is.  Readings: "top p %" = floor(p n / 100) vertices, at
 * least one; the fit takes every k >= 5 with at least one vertex,
 * unweighted, and fails with fewer than two such k (gamma = R^2 = NaN). */
typedef struct blest_degree_report {
    double top1;          /* share of the total degree held by the top 1 % */
    double top10;         /* share held by the top 10 % */
    double gamma;         /* minus the slope of the log-log histogram fit (NaN: no fit) */
    double r2;            /* R^2 of that fit (NaN: no fit) */
    int32_t points;       /* degrees k >= 5 present (fit points) */
    int32_t concentrated; /* test (a) */
    int32_t powerlaw;     /* test (b) */
    int32_t heavy;        /* (a) or (b) */
} blest_degree_report;

typedef struct blest_scale_free_report {
    blest_degree_report out_deg;
    blest_degree_report in_deg;   /* equals out_deg when in_deg was NULL */
    int32_t scale_free;           /* out_deg.heavy or in_deg.heavy */
} blest_scale_free_report;

/* Run the test on caller degree arrays (n int32 each, host or device;
 * in_deg NULL for an undirected graph).  The histogram is built on the GPU.
 * INVALID for n < 1, n >= 2^31 or a negative degree. */
blest_status blest_scale_free_test(const int32_t *out_deg, const int32_t *in_deg, int64_t n,
                                   blest_scale_free_report *out);

/* Test hook for the timed-out grid barrier: launches a cooperative kernel in
 * which one block waits on a barrier no other block joins.  Returns
 * BLEST_ERR_TIMEOUT after about timeout_ms when the wait gives up as it
 * should; the context stays usable. */
blest_status blest_selftest_barrier_timeout(int32_t timeout_ms);

#ifdef __cplusplus
}
#endif
#endif /* BLEST_H */
