// Vertex reordering on the device (§4): reverse Cuthill-McKee (§4.2) and
// JaccardWithWindows (§4.1, Algorithm 1).
#pragma once
#include "handle.h"

// Computes new_of_old (n entries, a permutation of [0, n)) for the graph
// (rp, col) according to o->reorder; *applied receives the ordering used
// (AUTO resolves to RCM or JACCARD).
blest_status reorder_graph(blest_graph *h, const long long *rp, const int *col, int64_t n, int64_t nnz,
                           const blest_build_opts *o, int *new_of_old, int *applied);
