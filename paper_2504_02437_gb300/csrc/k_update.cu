// Loss (Eq. 10-11, Section 3.2 "Map Optimization") and the Adam update.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ float block_sum(float v, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < kRedThreads / 32; ++k) t += sh[k];
    return t;   // valid in thread 0
}

// L1 photometric term: per-block partial sums of |C - I| (each view's sum is
// scaled by lambda_color / 3HW), and dL/dC = lambda_color sign(C - I) / 3HW.
__global__ void __launch_bounds__(kRedThreads) k_l1(const float* __restrict__ rgb, const float* __restrict__ tgt,
                                                    size_t total, float scale, float* __restrict__ dLdC,
                                                    float* __restrict__ partials) {
    __shared__ float sh[kRedThreads / 32];
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)kRedThreads + threadIdx.x; i < total; i += (size_t)gridDim.x * kRedThreads) {
        float r = rgb[i] - tgt[i];
        acc += fabsf(r);
        dLdC[i] = scale * (float)((r > 0.f) - (r < 0.f));
    }
    float t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t * scale;
}

// Planar term of Eq. 10: partial sums of max(floor, min_k exp(log-scale_k)).
__global__ void __launch_bounds__(kRedThreads) k_planar(const float* __restrict__ P, int n, int cap, float floor_,
                                                        float scale, float* __restrict__ partials) {
    __shared__ float sh[kRedThreads / 32];
    float acc = 0.f;
    for (int i = blockIdx.x * kRedThreads + threadIdx.x; i < n; i += gridDim.x * kRedThreads) {
        float s0 = expf(P[3 * (size_t)cap + i]), s1 = expf(P[4 * (size_t)cap + i]), s2 = expf(P[5 * (size_t)cap + i]);
        acc += fmaxf(floor_, fminf(s0, fminf(s1, s2)));
    }
    float t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t * scale;
}

// Fixed-order final reduction: out = {photometric + planar, photometric, planar}.
__global__ void __launch_bounds__(32) k_loss_final(const float* __restrict__ partials, int n_img, int n_reg,
                                                   float* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n_img; i += 32) a += partials[i];
    for (int i = threadIdx.x; i < n_reg; i += 32) b += partials[n_img + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
    }
    if (threadIdx.x == 0) {
        out[0] = (float)(a + b);
        out[1] = (float)a;
        out[2] = (float)b;
    }
}

struct AdamArgs {
    float lr[kParamRows];
    float b1, b2, eps, bc1, bc2;
};

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ P, const float* __restrict__ G,
                                              float* __restrict__ M, float* __restrict__ V, int n, int cap,
                                              AdamArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (i >= n) return;
    size_t k = (size_t)row * cap + i;
    float g = G[k];
    float m = a.b1 * M[k] + (1.f - a.b1) * g;
    float v = a.b2 * V[k] + (1.f - a.b2) * g * g;
    M[k] = m;
    V[k] = v;
    float mh = m / a.bc1, vh = v / a.bc2;
    P[k] -= a.lr[row] * mh / (sqrtf(vh) + a.eps);
}

}  // namespace

cudaError_t launch_loss(gs_ctx* c, const DevConst& k, const float* rgb, const float* target, float* loss_out,
                        cudaStream_t s) {
    const size_t HW = (size_t)c->width * c->height;
    const size_t total = (size_t)c->n_views * 3 * HW;
    const int nb_img = c->n_partials / 2, nb_reg = c->n_partials / 2;
    const float scale = k.lambda_color / (float)(3 * HW);
    c->launches += 3;
    k_l1<<<nb_img, kRedThreads, 0, s>>>(rgb, target, total, scale, c->dLdC, c->partials);
    k_planar<<<nb_reg, kRedThreads, 0, s>>>(c->params, c->n, c->cap, k.reg_floor,
                                            c->n > 0 ? k.lambda_reg / (float)c->n : 0.f, c->partials + nb_img);
    k_loss_final<<<1, 32, 0, s>>>(c->partials, nb_img, nb_reg, loss_out);
    return cudaGetLastError();
}

cudaError_t launch_adam(gs_ctx* c, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    AdamArgs a;
    static const int group[kParamRows] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3, 4, 4, 4};
    for (int r = 0; r < kParamRows; ++r) a.lr[r] = c->cfg.lr[group[r]];
    a.b1 = c->cfg.beta1;
    a.b2 = c->cfg.beta2;
    a.eps = c->cfg.eps;
    // bias corrections of step t (computed in double on the host)
    double t = (double)c->adam_t;
    a.bc1 = (float)(1.0 - pow((double)c->cfg.beta1, t));
    a.bc2 = (float)(1.0 - pow((double)c->cfg.beta2, t));
    dim3 grid((c->n + 255) / 256, kParamRows);
    ++c->launches;
    k_adam<<<grid, 256, 0, s>>>(c->params, c->grads, c->adam_m, c->adam_v, c->n, c->cap, a);
    return cudaGetLastError();
}

cudaError_t launch_copy_T(gs_ctx* c, float* T_out, cudaStream_t s) {
    if (T_out == nullptr) return cudaSuccess;
    return cudaMemcpyAsync(T_out, c->T_final, sizeof(float) * (size_t)c->n_views * c->width * c->height,
                           cudaMemcpyDeviceToDevice, s);
}

}  // namespace gs
