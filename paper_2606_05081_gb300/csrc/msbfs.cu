#include "msbfs.h"

void msbfs_release(blest_graph *h) { (void)h; }

extern "C" blest_status blest_msbfs(blest_handle h, const int32_t *sources, int32_t k, int32_t *levels) {
    (void)h; (void)sources; (void)k; (void)levels;
    return BLEST_ERR_UNSUPPORTED;
}
extern "C" blest_status blest_closeness(blest_handle h, int64_t *far, double *cc, int64_t *reach) {
    (void)h; (void)far; (void)cc; (void)reach;
    return BLEST_ERR_UNSUPPORTED;
}
extern "C" blest_status blest_build_many(int32_t g, const int64_t *vtx_off, const int64_t *edge_off,
                                         const int64_t *row_ptr, const int32_t *col_idx_local,
                                         const blest_build_opts *opts, blest_handle *out) {
    (void)g; (void)vtx_off; (void)edge_off; (void)row_ptr; (void)col_idx_local; (void)opts; (void)out;
    return BLEST_ERR_UNSUPPORTED;
}
extern "C" blest_status blest_bfs_many(blest_handle h, const int32_t *sources, int32_t *levels) {
    (void)h; (void)sources; (void)levels;
    return BLEST_ERR_UNSUPPORTED;
}
