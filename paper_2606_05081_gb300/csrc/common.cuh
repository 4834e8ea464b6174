// Shared device helpers for the BVSS BFS kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/blest.h"

#define FULL_MASK 0xFFFFFFFFu

#define CUDA_TRY(expr)                                                      \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) {                                            \
            blest_internal_record_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return (_e == cudaErrorMemoryAllocation) ? BLEST_ERR_OOM : BLEST_ERR_CUDA; \
        }                                                                   \
    } while (0)

extern "C" void blest_internal_record_cuda_error(cudaError_t e, const char *expr, const char *file,
                                                 int line);

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

// Fire-and-forget atomic OR (the return value is never consumed, so the
// memory system may complete it asynchronously: §5.2).
__device__ __forceinline__ void red_or(unsigned *p, unsigned v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    return x;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    return x;
}

// Control block of one persistent launch.  Counter slots form a ring of 4 so
// that one grid barrier per top-down level suffices (see bfs.cu).
struct Ctl {
    unsigned long long bar;  // grid-barrier arrivals (monotone within a launch)
    int err;               // device status (blest_status); 0 = OK
    int nlevels;           // levels run (written by block 0)
    int timeout_where;     // barrier index that timed out
    int qlen[4];           // VSS queue length per level slot
    int sqlen[4];          // slice-set queue length per level slot
    unsigned long long newv[4];    // vertices discovered per level slot
    unsigned long long fedges[4];  // out-arcs of those vertices
    unsigned long long scan_v[4];  // bottom-up: vertices probed
    unsigned long long scan_a[4];  // bottom-up: in-neighbour ids read
    int xq[4];             // entries written so far when a deferred VSS queue is expanded
};

// Timed-out grid barrier for a cooperative launch.  Every block calls it the
// same number of times.  Arrivals are counted on a monotone counter; the
// k-th barrier waits for k*gridDim.x arrivals.  A wait that exceeds the
// budget records BLEST_ERR_TIMEOUT and returns; once err is set every block
// leaves at its next barrier (whose spin loop checks err every 64 polls), so
// no block spins forever.
// Returns true when the grid may proceed.
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, unsigned &epoch, uint64_t budget_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        const unsigned long long target = (unsigned long long)epoch * gridDim.x;
        // release: the block's writes (ordered before by bar.sync) become visible
        // no later than the arrival; the acquire loads below order what follows
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(&ctl->bar), "l"(1ull) : "memory");
        const uint64_t t0 = global_ns();
        int ok = 1;
        unsigned spins = 0;
        while (ld_acquire_u64(&ctl->bar) < target) {
            if ((++spins & 63u) == 0) {
                if (ld_volatile_i32(&ctl->err) != 0) { ok = 0; break; }
                if (global_ns() - t0 > budget_ns) {
                    atomicCAS(&ctl->err, 0, (int)BLEST_ERR_TIMEOUT);
                    atomicCAS(&ctl->timeout_where, 0, (int)epoch);
                    ok = 0;
                    break;
                }
            }
            if (spins > 256) __nanosleep(32);
        }
        // no error check once the barrier has completed: a block that gave up
        // had arrived first, so the others finish this barrier and see the
        // error in the spin loop of the next one
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
