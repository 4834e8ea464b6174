// Learned per-level kernel choice: a 3-layer MLP (6 -> 32 -> 32 -> 9, tanh
// hidden units, fp32) that predicts the log device time of each level
// choice -- a level mode and, for lazy top-down levels, the VSS passes a
// warp keeps in flight; the level runs the choice with the smallest
// prediction.  The same weights are trained on the device by mlp.cu.
//
// Choices: 0-4 are the level modes (BLEST_MODE_*), lazy ones with one pass
// in flight; 5, 6 = lazy CUDA-core with 2, 4 passes; 7, 8 = lazy b1-MMA
// with 2, 4 passes.
//
// Weight vector layout (fp32, MLP_NW values):
//   [0, 6)        feature means          [6, 12)      feature 1/std
//   W1 [32][6]    b1 [32]                W2 [32][32]  b2 [32]
//   W3 [9][32]    b3 [9]
// Features, in order: log1p(frontier vertices), log1p(frontier out-arcs),
// log1p(unvisited vertices), log1p(active BVSS slots = tau * |Q|),
// log1p(level index), log1p(average degree).
#pragma once
#include <cuda_runtime.h>

#define MLP_IN 6
#define MLP_H 32
#define MLP_OUT 9
#define MLP_OFF_MEAN 0
#define MLP_OFF_ISTD 6
#define MLP_OFF_W1 12
#define MLP_OFF_B1 (MLP_OFF_W1 + MLP_H * MLP_IN)
#define MLP_OFF_W2 (MLP_OFF_B1 + MLP_H)
#define MLP_OFF_B2 (MLP_OFF_W2 + MLP_H * MLP_H)
#define MLP_OFF_W3 (MLP_OFF_B2 + MLP_H)
#define MLP_OFF_B3 (MLP_OFF_W3 + MLP_OUT * MLP_H)
#define MLP_NW (MLP_OFF_B3 + MLP_OUT)

__host__ __device__ inline void mlp_raw_features(float *x, long long frontier, long long fedges,
                                                 long long unvisited, long long slots, int level,
                                                 float avg_deg) {
    x[0] = log1pf((float)frontier);
    x[1] = log1pf((float)fedges);
    x[2] = log1pf((float)(unvisited > 0 ? unvisited : 0));
    x[3] = log1pf((float)slots);
    x[4] = log1pf((float)level);
    x[5] = log1pf(avg_deg);
}

// Shared-memory copy of the weights for the warp-cooperative forward pass:
// the same MLP_NW values with W1, W2 and W3 stored transposed (input-major),
// so the lanes of a warp read consecutive words (no bank conflicts).  Called
// by every thread of the block; the caller synchronises afterwards.
__device__ __forceinline__ void mlp_stage_weights(const float *__restrict__ w, float *s) {
    for (int i = threadIdx.x; i < MLP_NW; i += blockDim.x) {
        int d = i;
        if (i >= MLP_OFF_W1 && i < MLP_OFF_B1) {            // W1[h][k] -> [k][h]
            const int r = (i - MLP_OFF_W1) / MLP_IN, c = (i - MLP_OFF_W1) % MLP_IN;
            d = MLP_OFF_W1 + c * MLP_H + r;
        } else if (i >= MLP_OFF_W2 && i < MLP_OFF_B2) {     // W2[h][k] -> [k][h]
            const int r = (i - MLP_OFF_W2) / MLP_H, c = (i - MLP_OFF_W2) % MLP_H;
            d = MLP_OFF_W2 + c * MLP_H + r;
        } else if (i >= MLP_OFF_W3 && i < MLP_OFF_B3) {     // W3[o][k] -> [k][o]
            const int r = (i - MLP_OFF_W3) / MLP_H, c = (i - MLP_OFF_W3) % MLP_H;
            d = MLP_OFF_W3 + c * MLP_OUT + r;
        }
        s[d] = w[i];
    }
}

// Warp-cooperative forward pass on raw features x (all 32 lanes call it;
// lane h owns hidden unit h of both layers), weights staged by
// mlp_stage_weights.  Lane o < MLP_OUT returns the prediction for mode o
// (other lanes return 0).
__device__ __forceinline__ float mlp_forward_warp(const float *__restrict__ w, const float *xr) {
    const int lane = threadIdx.x & 31;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = (xr[i] - w[MLP_OFF_MEAN + i]) * w[MLP_OFF_ISTD + i];
    float a1 = w[MLP_OFF_B1 + lane];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) a1 = fmaf(w[MLP_OFF_W1 + i * MLP_H + lane], x[i], a1);
    const float h1 = tanhf(a1);
    // four interleaved partial sums (inputs k = j mod 4) shorten the chain of
    // dependent multiply-adds the level start waits on; summed in a fixed order
    float p2[4] = {w[MLP_OFF_B2 + lane], 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < MLP_H; ++k)
        p2[k & 3] = fmaf(w[MLP_OFF_W2 + k * MLP_H + lane], __shfl_sync(0xFFFFFFFFu, h1, k), p2[k & 3]);
    const float h2 = tanhf((p2[0] + p2[1]) + (p2[2] + p2[3]));
    const int o = lane < MLP_OUT ? lane : 0;
    float p3[4] = {w[MLP_OFF_B3 + o], 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < MLP_H; ++k)
        p3[k & 3] = fmaf(w[MLP_OFF_W3 + k * MLP_OUT + o], __shfl_sync(0xFFFFFFFFu, h2, k), p3[k & 3]);
    const float y = (p3[0] + p3[1]) + (p3[2] + p3[3]);
    return lane < MLP_OUT ? y : 0.f;
}

// Bottom-up guard: a bottom-up level reads every unvisited vertex, a
// top-down level the frontier's out-arcs, so a level with more than 16
// unvisited vertices per frontier arc never runs bottom-up whatever the
// network predicts (this keeps graphs unlike the training set away from
// the one choice whose cost grows with the unvisited set; scheduled slots
// would overstate the top-down work where VSSs are mostly padding).
// Tested on the raw features: log1p(unvisited) > log1p(frontier arcs) +
// log(16).
#define MLP_BU_GUARD_LOG 2.7725887f

__host__ __device__ inline bool mlp_bu_blocked(const float *xraw) { return xraw[2] > xraw[1] + MLP_BU_GUARD_LOG; }

// argmin over the MLP_OUT predictions (lowest index on ties), skipping
// bottom-up (choice 4) when blocked; all lanes get it
__device__ __forceinline__ int mlp_argmin_warp(float y, bool no_bu) {
    int arg = -1;
    float best = 0.f;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        const float v = __shfl_sync(0xFFFFFFFFu, y, o);
        if (no_bu && o == 4) continue;
        if (arg < 0 || v < best) { best = v; arg = o; }
    }
    return arg;
}

// Called by all 32 lanes of one warp; every lane returns the chosen mode.
__device__ __forceinline__ int mlp_choose_warp(const float *__restrict__ w, long long frontier, long long fedges,
                                               long long unvisited, long long slots, int level, float avg_deg) {
    float x[MLP_IN];
    mlp_raw_features(x, frontier, fedges, unvisited, slots, level, avg_deg);
    return mlp_argmin_warp(mlp_forward_warp(w, x), mlp_bu_blocked(x));
}

// mode and VSS passes in flight of a choice (launch_batch for the rule's and
// fixed modes, which use the launch's setting)
__host__ __device__ inline int mlp_choice_mode(int c) { return c < 5 ? c : (c < 7 ? 2 : 3); }
__host__ __device__ inline int mlp_choice_batch(int c) { return c < 5 ? 1 : ((c - 5) % 2 == 0 ? 2 : 4); }
