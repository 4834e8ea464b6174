// Device-wide primitives used by the graph builder: exclusive scan and a
// stable LSD radix sort of 64-bit keys with optional 32-bit payloads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Exclusive scan of n int64 values into out[0..n]; out[n] receives the total.
// in may equal out.  tmp must hold scan_tmp_elems(n) int64.
size_t scan_tmp_elems(int64_t n);
cudaError_t scan_exclusive_i64(const long long *in, long long *out, int64_t n, long long *tmp,
                               cudaStream_t st);
// Same for int32 inputs (converted to int64 on the fly).
cudaError_t scan_exclusive_i32_to_i64(const int *in, long long *out, int64_t n, long long *tmp,
                                      cudaStream_t st);

// Stable LSD radix sort of keys (and vals if non-null) on bits [0, key_bits).
// keys/vals are sorted in place; kalt/valt are scratch of n elements;
// hist must hold radix_hist_elems(n) int64.
size_t radix_hist_elems(int64_t n);
cudaError_t radix_sort_u64(unsigned long long *keys, unsigned *vals, unsigned long long *kalt,
                           unsigned *valt, int64_t n, int key_bits, long long *hist,
                           long long *scan_tmp, cudaStream_t st);

static inline int ceil_log2_i64(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}
