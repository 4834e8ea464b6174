// Multi-source BFS (§6.1, Algorithm 5), closeness (§6.2) and batched small
// graphs: host entry points implemented in msbfs.cu and many.cu.
#pragma once
#include "handle.h"

void msbfs_release(blest_graph *h);
void many_release(blest_graph *h);
