// Training and evaluation of the level-mode MLP on the device.
//
// Full-batch training with Adam.  Per epoch:
//   k_mlp_forward   one thread per sample: normalised inputs, both hidden
//                   layers, the five predictions, the masked squared error
//                   and the back-propagated activations (dY, dA2, dA1), all
//                   stored feature-major so the next kernel reads them
//                   coalesced;
//   k_mlp_grad      one warp per parameter: the gradient is a dot product
//                   over the samples, summed by each lane in sample order and
//                   then by a fixed shuffle tree, so training is bit-for-bit
//                   deterministic (no atomics);
//   k_mlp_adam      one thread per parameter (normalisation entries frozen).
// The arithmetic of the forward pass (fmaf chains in the same order, tanhf)
// is that of the in-kernel inference in mlp.h.
#include <cstring>
#include <vector>

#include "handle.h"
#include "mlp.h"

namespace {

struct Bufs {
    float *X, *T, *M;          // [6][N], [5][N], [5][N]   (feature-major)
    float *XN, *H1, *H2;       // [6][N], [32][N], [32][N]
    float *DY, *DA2, *DA1;     // [5][N], [32][N], [32][N]
    float *SE;                 // [N] per-sample squared error (masked)
    float *W, *G, *Mom, *Vel;  // [NW]
    float *loss;               // [1]
};

__global__ void k_mlp_forward(Bufs B, int n, float inv_cnt) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float *w = B.W;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) {
        x[i] = (B.X[(size_t)i * n + s] - w[MLP_OFF_MEAN + i]) * w[MLP_OFF_ISTD + i];
        B.XN[(size_t)i * n + s] = x[i];
    }
    float h1[MLP_H], h2[MLP_H];
#pragma unroll 4
    for (int h = 0; h < MLP_H; ++h) {
        float a = w[MLP_OFF_B1 + h];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) a = fmaf(w[MLP_OFF_W1 + h * MLP_IN + i], x[i], a);
        h1[h] = tanhf(a);
        B.H1[(size_t)h * n + s] = h1[h];
    }
#pragma unroll 2
    for (int h = 0; h < MLP_H; ++h) {
        float a = w[MLP_OFF_B2 + h];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) a = fmaf(w[MLP_OFF_W2 + h * MLP_H + k], h1[k], a);
        h2[h] = tanhf(a);
        B.H2[(size_t)h * n + s] = h2[h];
    }
    float dy[MLP_OUT];
    float se = 0.f;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        float y = w[MLP_OFF_B3 + o];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) y = fmaf(w[MLP_OFF_W3 + o * MLP_H + k], h2[k], y);
        const float m = B.M[(size_t)o * n + s];
        const float r = (y - B.T[(size_t)o * n + s]) * m;
        se += r * r;
        dy[o] = 2.f * r * inv_cnt;
        B.DY[(size_t)o * n + s] = dy[o];
    }
    B.SE[s] = se;
    // dA2 = (dY W3) * (1 - h2^2)
    float da2[MLP_H];
#pragma unroll 4
    for (int k = 0; k < MLP_H; ++k) {
        float a = 0.f;
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) a = fmaf(dy[o], w[MLP_OFF_W3 + o * MLP_H + k], a);
        da2[k] = a * (1.f - h2[k] * h2[k]);
        B.DA2[(size_t)k * n + s] = da2[k];
    }
    // dA1 = (dA2 W2) * (1 - h1^2)
#pragma unroll 2
    for (int k = 0; k < MLP_H; ++k) {
        float a = 0.f;
#pragma unroll
        for (int h = 0; h < MLP_H; ++h) a = fmaf(da2[h], w[MLP_OFF_W2 + h * MLP_H + k], a);
        B.DA1[(size_t)k * n + s] = a * (1.f - h1[k] * h1[k]);
    }
}

// fixed-order warp sum of a[i] * b[i] over i < n (b == nullptr: sum of a)
__device__ __forceinline__ float warp_dot(const float *a, const float *b, int n) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
    for (int i = lane; i < n; i += 32) acc = b ? fmaf(a[i], b[i], acc) : acc + a[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    return acc;
}

__global__ void k_mlp_grad(Bufs B, int n) {
    const int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);   // parameter index
    if (p >= MLP_NW) return;
    float g = 0.f;
    if (p < MLP_OFF_W1) {
        g = 0.f;
    } else if (p < MLP_OFF_B1) {
        const int h = (p - MLP_OFF_W1) / MLP_IN, i = (p - MLP_OFF_W1) % MLP_IN;
        g = warp_dot(B.DA1 + (size_t)h * n, B.XN + (size_t)i * n, n);
    } else if (p < MLP_OFF_W2) {
        g = warp_dot(B.DA1 + (size_t)(p - MLP_OFF_B1) * n, nullptr, n);
    } else if (p < MLP_OFF_B2) {
        const int h = (p - MLP_OFF_W2) / MLP_H, k = (p - MLP_OFF_W2) % MLP_H;
        g = warp_dot(B.DA2 + (size_t)h * n, B.H1 + (size_t)k * n, n);
    } else if (p < MLP_OFF_W3) {
        g = warp_dot(B.DA2 + (size_t)(p - MLP_OFF_B2) * n, nullptr, n);
    } else if (p < MLP_OFF_B3) {
        const int o = (p - MLP_OFF_W3) / MLP_H, k = (p - MLP_OFF_W3) % MLP_H;
        g = warp_dot(B.DY + (size_t)o * n, B.H2 + (size_t)k * n, n);
    } else {
        g = warp_dot(B.DY + (size_t)(p - MLP_OFF_B3) * n, nullptr, n);
    }
    if ((threadIdx.x & 31) == 0) B.G[p] = g;
    if (p == 0) {
        const float l = warp_dot(B.SE, nullptr, n);
        if ((threadIdx.x & 31) == 0) B.loss[0] = l;
    }
}

__global__ void k_mlp_adam(Bufs B, int t, float lr, float b1, float b2, float eps, float wd) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NW || p < MLP_OFF_W1) return;
    const float g = B.G[p] + wd * B.W[p];   // L2 penalty (wd/2)|w|^2
    const float m = b1 * B.Mom[p] + (1.f - b1) * g;
    const float v = b2 * B.Vel[p] + (1.f - b2) * g * g;
    B.Mom[p] = m;
    B.Vel[p] = v;
    const float mh = m / (1.f - powf(b1, (float)t));
    const float vh = v / (1.f - powf(b2, (float)t));
    B.W[p] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_mlp_features(const blest_level_log *__restrict__ recs, int n, float avg_deg, float *out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[MLP_IN];
    const blest_level_log r = recs[s];
    mlp_raw_features(x, r.frontier, r.frontier_edges, r.unvisited, r.slots, r.level, avg_deg);
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) out[(size_t)s * MLP_IN + i] = x[i];
}

// one warp per sample, the in-kernel inference routine itself (weights
// staged in shared memory exactly as the BFS kernel stages them)
__global__ void k_mlp_predict(const float *__restrict__ w, const float *__restrict__ feats, int n, float *pred,
                              int *choice) {
    __shared__ float sw[MLP_NW];
    mlp_stage_weights(w, sw);
    __syncthreads();
    w = sw;
    const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (s >= n) return;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = feats[(size_t)s * MLP_IN + i];
    const float y = mlp_forward_warp(w, x);
    const int lane = threadIdx.x & 31;
    if (pred && lane < MLP_OUT) pred[(size_t)s * MLP_OUT + lane] = y;
    const int c = mlp_argmin_warp(y, mlp_bu_blocked(x));
    if (choice && lane == 0) choice[s] = c;
}

// ---- host helpers
struct DevSet {
    Bufs b;
    std::vector<void *> ptrs;
    bool bad = false;
    float *get(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, count * sizeof(float) + 16) != cudaSuccess) { bad = true; return nullptr; }
        ptrs.push_back(p);
        return (float *)p;
    }
    ~DevSet() {
        for (void *p : ptrs) cudaFree(p);
    }
};

// Upload row-major host/device arrays [n][k] into feature-major device arrays.
blest_status upload_fm(const float *src, int64_t n, int k, float *dst) {
    std::vector<float> h((size_t)n * k), t((size_t)n * k);
    if (cudaMemcpy(h.data(), src, (size_t)n * k * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    for (int64_t s = 0; s < n; ++s)
        for (int i = 0; i < k; ++i) t[(size_t)i * n + s] = h[(size_t)s * k + i];
    return cudaMemcpy(dst, t.data(), (size_t)n * k * 4, cudaMemcpyHostToDevice) == cudaSuccess ? BLEST_OK
                                                                                               : BLEST_ERR_CUDA;
}

blest_status setup(DevSet &D, const float *features, const float *targets, const float *mask, int64_t n,
                   const float *weights, float *inv_cnt) {
    Bufs &B = D.b;
    B.X = D.get((size_t)n * MLP_IN);
    B.T = D.get((size_t)n * MLP_OUT);
    B.M = D.get((size_t)n * MLP_OUT);
    B.XN = D.get((size_t)n * MLP_IN);
    B.H1 = D.get((size_t)n * MLP_H);
    B.H2 = D.get((size_t)n * MLP_H);
    B.DY = D.get((size_t)n * MLP_OUT);
    B.DA2 = D.get((size_t)n * MLP_H);
    B.DA1 = D.get((size_t)n * MLP_H);
    B.SE = D.get((size_t)n);
    B.W = D.get(MLP_NW);
    B.G = D.get(MLP_NW);
    B.Mom = D.get(MLP_NW);
    B.Vel = D.get(MLP_NW);
    B.loss = D.get(1);
    if (D.bad) return BLEST_ERR_OOM;
    blest_status st;
    if ((st = upload_fm(features, n, MLP_IN, B.X)) != BLEST_OK) return st;
    if ((st = upload_fm(targets, n, MLP_OUT, B.T)) != BLEST_OK) return st;
    if ((st = upload_fm(mask, n, MLP_OUT, B.M)) != BLEST_OK) return st;
    std::vector<float> mh((size_t)n * MLP_OUT);
    cudaMemcpy(mh.data(), B.M, mh.size() * 4, cudaMemcpyDeviceToHost);
    double cnt = 0;
    for (float v : mh) cnt += v;
    *inv_cnt = (float)(1.0 / (cnt > 0 ? cnt : 1.0));
    if (cudaMemcpy(B.W, weights, MLP_NW * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    cudaMemset(B.G, 0, MLP_NW * 4);
    cudaMemset(B.Mom, 0, MLP_NW * 4);
    cudaMemset(B.Vel, 0, MLP_NW * 4);
    return BLEST_OK;
}

}  // namespace

extern "C" blest_status blest_mlp_loss_grad(const float *features, const float *targets, const float *mask,
                                            int64_t n, const float *weights, float *loss, float *grad) {
    if (!features || !targets || !mask || !weights || n < 1 || n > (1 << 24)) return BLEST_ERR_INVALID;
    DevSet D;
    float inv_cnt = 1.f;
    blest_status st = setup(D, features, targets, mask, n, weights, &inv_cnt);
    if (st != BLEST_OK) return st;
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128>>>(D.b, (int)n, inv_cnt);
    k_mlp_grad<<<(MLP_NW * 32 + 255) / 256, 256>>>(D.b, (int)n);
    if (cudaDeviceSynchronize() != cudaSuccess) return BLEST_ERR_CUDA;
    float l = 0.f;
    cudaMemcpy(&l, D.b.loss, 4, cudaMemcpyDeviceToHost);
    if (loss) *loss = l * inv_cnt;
    if (grad && cudaMemcpy(grad, D.b.G, MLP_NW * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    return BLEST_OK;
}

extern "C" blest_status blest_mlp_train(const float *features, const float *targets, const float *mask, int64_t n,
                                        int32_t epochs, float lr, float weight_decay, float *weights,
                                        float *loss_out) {
    if (!features || !targets || !mask || !weights || n < 1 || n > (1 << 24) || epochs < 1 || epochs > 1000000 ||
        !(lr > 0.f) || !(weight_decay >= 0.f))
        return BLEST_ERR_INVALID;
    DevSet D;
    float inv_cnt = 1.f;
    blest_status st = setup(D, features, targets, mask, n, weights, &inv_cnt);
    if (st != BLEST_OK) return st;
    std::vector<float> lh;
    if (loss_out) lh.resize((size_t)epochs);
    for (int t = 1; t <= epochs; ++t) {
        k_mlp_forward<<<(unsigned)((n + 127) / 128), 128>>>(D.b, (int)n, inv_cnt);
        k_mlp_grad<<<(MLP_NW * 32 + 255) / 256, 256>>>(D.b, (int)n);
        k_mlp_adam<<<(MLP_NW + 255) / 256, 256>>>(D.b, t, lr, 0.9f, 0.999f, 1e-8f, weight_decay);
        if (loss_out) {
            float l = 0.f;
            cudaMemcpy(&l, D.b.loss, 4, cudaMemcpyDeviceToHost);   // loss before step t
            lh[(size_t)t - 1] = l * inv_cnt;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaMemcpy(weights, D.b.W, MLP_NW * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    if (loss_out && cudaMemcpy(loss_out, lh.data(), lh.size() * 4, cudaMemcpyDefault) != cudaSuccess)
        return BLEST_ERR_CUDA;
    return BLEST_OK;
}

extern "C" blest_status blest_mlp_features(const blest_level_log *recs, int64_t n, float avg_deg, float *out) {
    if (!recs || !out || n < 1 || n > (1 << 24)) return BLEST_ERR_INVALID;
    blest_level_log *dr = nullptr;
    float *df = nullptr;
    if (cudaMalloc(&dr, (size_t)n * sizeof(blest_level_log)) != cudaSuccess) return BLEST_ERR_OOM;
    if (cudaMalloc(&df, (size_t)n * MLP_IN * 4) != cudaSuccess) { cudaFree(dr); return BLEST_ERR_OOM; }
    cudaMemcpy(dr, recs, (size_t)n * sizeof(blest_level_log), cudaMemcpyDefault);
    k_mlp_features<<<(unsigned)((n + 127) / 128), 128>>>(dr, (int)n, avg_deg, df);
    cudaError_t e = cudaMemcpy(out, df, (size_t)n * MLP_IN * 4, cudaMemcpyDefault);
    cudaFree(dr);
    cudaFree(df);
    return e == cudaSuccess ? BLEST_OK : BLEST_ERR_CUDA;
}

extern "C" blest_status blest_mlp_predict(const float *weights, const float *features, int64_t n, float *pred,
                                          int32_t *choice) {
    if (!weights || !features || n < 1 || n > (1 << 24)) return BLEST_ERR_INVALID;
    float *dw = nullptr, *df = nullptr, *dp = nullptr;
    int *dc = nullptr;
    bool ok = cudaMalloc(&dw, MLP_NW * 4) == cudaSuccess && cudaMalloc(&df, (size_t)n * MLP_IN * 4) == cudaSuccess &&
              cudaMalloc(&dp, (size_t)n * MLP_OUT * 4) == cudaSuccess && cudaMalloc(&dc, (size_t)n * 4) == cudaSuccess;
    blest_status st = ok ? BLEST_OK : BLEST_ERR_OOM;
    if (ok) {
        cudaMemcpy(dw, weights, MLP_NW * 4, cudaMemcpyDefault);
        cudaMemcpy(df, features, (size_t)n * MLP_IN * 4, cudaMemcpyDefault);
        k_mlp_predict<<<(unsigned)((n * 32 + 255) / 256), 256>>>(dw, df, (int)n, dp, dc);
        if (cudaDeviceSynchronize() != cudaSuccess) st = BLEST_ERR_CUDA;
        if (st == BLEST_OK && pred) st = cudaMemcpy(pred, dp, (size_t)n * MLP_OUT * 4, cudaMemcpyDefault) == cudaSuccess ? st : BLEST_ERR_CUDA;
        if (st == BLEST_OK && choice) st = cudaMemcpy(choice, dc, (size_t)n * 4, cudaMemcpyDefault) == cudaSuccess ? st : BLEST_ERR_CUDA;
    }
    cudaFree(dw);
    cudaFree(df);
    cudaFree(dp);
    cudaFree(dc);
    return st;
}
