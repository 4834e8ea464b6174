#include "reorder.h"

blest_status reorder_graph(blest_graph *h, const long long *rp, const int *col, int64_t n, int64_t nnz,
                           const blest_build_opts *o, int *new_of_old, int *applied) {
    (void)h; (void)rp; (void)col; (void)n; (void)nnz; (void)o; (void)new_of_old; (void)applied;
    return BLEST_ERR_UNSUPPORTED;
}
