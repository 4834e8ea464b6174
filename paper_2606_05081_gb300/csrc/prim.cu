// Device-wide exclusive scan and stable LSD radix sort (build-time helpers).
#include "common.cuh"
#include "prim.cuh"

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename In>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const In *__restrict__ in, long long *sums,
                                                               int64_t n) {
    __shared__ long long warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long acc = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) acc += (long long)in[k];
    }
    acc = warp_sum(acc);
    if (lane_id() == 0) warp_tot[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long v = threadIdx.x < SCAN_THREADS / 32 ? warp_tot[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// Exclusive scan of one tile plus a tile offset; writes out[n] = total when
// the tile holds the last element.
template <typename In>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const In *in, long long *out,
                                                             const long long *tile_off, int64_t n) {
    __shared__ long long warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS];
    long long run = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t k = base + i;
        v[i] = (k < n) ? (long long)in[k] : 0;
        run += v[i];
    }
    // exclusive prefix of per-thread sums across the block
    long long incl = warp_incl_scan(run);
    if (lane_id() == 31) warp_tot[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long w = threadIdx.x < SCAN_THREADS / 32 ? warp_tot[threadIdx.x] : 0;
        long long wi = warp_incl_scan(w);
        if (threadIdx.x < SCAN_THREADS / 32) warp_tot[threadIdx.x] = wi - w;
    }
    __syncthreads();
    long long off = (tile_off ? tile_off[blockIdx.x] : 0) + warp_tot[threadIdx.x >> 5] + (incl - run);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t k = base + i;
        if (k < n) out[k] = off;
        if (k == n - 1) out[n] = off + v[i];
        off += v[i];
    }
    if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

template <typename In>
cudaError_t scan_impl(const In *in, long long *out, int64_t n, long long *tmp, cudaStream_t st) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) {
        k_tile_scan<In><<<1, SCAN_THREADS, 0, st>>>(in, out, nullptr, n);
        return cudaGetLastError();
    }
    long long *sums = tmp;            // tiles + 1
    long long *rest = tmp + tiles + 1;
    k_tile_reduce<In><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, sums, n);
    cudaError_t e = scan_impl<long long>(sums, sums, tiles, rest, st);
    if (e != cudaSuccess) return e;
    k_tile_scan<In><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, out, sums, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------ radix sort
constexpr int RS_WARPS = 8;
constexpr int RS_ITEMS = 128;              // rounds of 32 per warp tile
constexpr int RS_TILE = 32 * RS_ITEMS;     // items per warp tile
constexpr int RS_BITS = 8;
constexpr int RS_BINS = 1 << RS_BITS;

__global__ void __launch_bounds__(RS_WARPS * 32) k_rs_hist(const unsigned long long *__restrict__ keys,
                                                           int64_t n, int shift, int64_t ntiles,
                                                           long long *hist) {
    __shared__ int cnt[RS_WARPS][RS_BINS];
    const int w = threadIdx.x >> 5, lane = lane_id();
    for (int i = lane; i < RS_BINS; i += 32) cnt[w][i] = 0;
    __syncwarp();
    const int64_t tile = (int64_t)blockIdx.x * RS_WARPS + w;
    if (tile < ntiles) {
        const int64_t base = tile * RS_TILE;
        for (int r = 0; r < RS_ITEMS; ++r) {
            int64_t k = base + r * 32 + lane;
            if (k < n) atomicAdd(&cnt[w][(keys[k] >> shift) & (RS_BINS - 1)], 1);
        }
    }
    __syncwarp();
    if (tile < ntiles)
        for (int i = lane; i < RS_BINS; i += 32) hist[(int64_t)i * ntiles + tile] = cnt[w][i];
}

__global__ void __launch_bounds__(RS_WARPS * 32) k_rs_scatter(
    const unsigned long long *__restrict__ kin, const unsigned *__restrict__ vin, unsigned long long *kout,
    unsigned *vout, int64_t n, int shift, int64_t ntiles, const long long *__restrict__ off) {
    __shared__ long long pos[RS_WARPS][RS_BINS];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int64_t tile = (int64_t)blockIdx.x * RS_WARPS + w;
    if (tile >= ntiles) return;
    for (int i = lane; i < RS_BINS; i += 32) pos[w][i] = off[(int64_t)i * ntiles + tile];
    __syncwarp();
    const unsigned lt = lanemask_lt();
    const int64_t base = tile * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t k = base + r * 32 + lane;
        const bool ok = k < n;
        unsigned long long key = ok ? kin[k] : 0ull;
        int d = ok ? (int)((key >> shift) & (RS_BINS - 1)) : RS_BINS; // RS_BINS = dummy group
        unsigned peers = __match_any_sync(FULL_MASK, d);
        int rank = __popc(peers & lt);
        long long p = ok ? pos[w][d] + rank : 0;
        __syncwarp();
        if (ok && rank == 0) pos[w][d] += __popc(peers);
        __syncwarp();
        if (ok) {
            kout[p] = key;
            if (vin) vout[p] = vin[k];
        }
    }
}

}  // namespace

size_t scan_tmp_elems(int64_t n) {
    size_t tot = 0;
    int64_t t = (n + SCAN_TILE - 1) / SCAN_TILE;
    while (t > 1) {
        tot += (size_t)t + 1;
        t = (t + SCAN_TILE - 1) / SCAN_TILE;
    }
    return tot + 2;
}

cudaError_t scan_exclusive_i64(const long long *in, long long *out, int64_t n, long long *tmp,
                               cudaStream_t st) {
    return scan_impl<long long>(in, out, n, tmp, st);
}
cudaError_t scan_exclusive_i32_to_i64(const int *in, long long *out, int64_t n, long long *tmp,
                                      cudaStream_t st) {
    return scan_impl<int>(in, out, n, tmp, st);
}

size_t radix_hist_elems(int64_t n) {
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles < 1) ntiles = 1;
    return (size_t)ntiles * RS_BINS + 1;
}

cudaError_t radix_sort_u64(unsigned long long *keys, unsigned *vals, unsigned long long *kalt,
                           unsigned *valt, int64_t n, int key_bits, long long *hist,
                           long long *scan_tmp, cudaStream_t st) {
    if (n <= 1 || key_bits <= 0) return cudaSuccess;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const unsigned blocks = (unsigned)((ntiles + RS_WARPS - 1) / RS_WARPS);
    unsigned long long *ka = keys, *kb = kalt;
    unsigned *va = vals, *vb = valt;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += RS_BITS) {
        k_rs_hist<<<blocks, RS_WARPS * 32, 0, st>>>(ka, n, shift, ntiles, hist);
        cudaError_t e = scan_exclusive_i64(hist, hist, ntiles * RS_BINS, scan_tmp, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<blocks, RS_WARPS * 32, 0, st>>>(ka, va, kb, vb, n, shift, ntiles, hist);
        unsigned long long *t = ka; ka = kb; kb = t;
        unsigned *tv = va; va = vb; vb = tv;
        ++passes;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
        if (vals) cudaMemcpyAsync(vals, va, (size_t)n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}
