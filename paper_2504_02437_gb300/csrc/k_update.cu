// Loss (Eq. 10-11, Section 3.2 "Map Optimization") and the Adam update.
#include <algorithm>

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

// L1 photometric term: per-block partial sums of |C - I| (scaled by
// lambda_color / 3HW), and dL/dC = lambda_color sign(C - I) / 3HW. Vectorised
// by float4 over the flat [V][3][H][W] arrays; `total` is a multiple of 4 here
// and the tail (if any) is handled by the scalar loop.
__global__ void __launch_bounds__(kRedThreads) k_l1(const float* __restrict__ rgb, const float* __restrict__ tgt,
                                                    size_t total, float scale, float* __restrict__ dLdC,
                                                    float* __restrict__ partials) {
    __shared__ float sh[kRedThreads / 32];
    float acc = 0.f;
    const size_t n4 = total / 4;
    const size_t stride = (size_t)gridDim.x * kRedThreads;
    const float4* r4 = reinterpret_cast<const float4*>(rgb);
    const float4* t4 = reinterpret_cast<const float4*>(tgt);
    float4* d4 = reinterpret_cast<float4*>(dLdC);
    for (size_t i = blockIdx.x * (size_t)kRedThreads + threadIdx.x; i < n4; i += stride) {
        const float4 a = r4[i], b = t4[i];
        const float rx = a.x - b.x, ry = a.y - b.y, rz = a.z - b.z, rw = a.w - b.w;
        acc += (fabsf(rx) + fabsf(ry)) + (fabsf(rz) + fabsf(rw));
        d4[i] = make_float4(scale * (float)((rx > 0.f) - (rx < 0.f)), scale * (float)((ry > 0.f) - (ry < 0.f)),
                            scale * (float)((rz > 0.f) - (rz < 0.f)), scale * (float)((rw > 0.f) - (rw < 0.f)));
    }
    for (size_t i = 4 * n4 + blockIdx.x * (size_t)kRedThreads + threadIdx.x; i < total; i += stride) {
        const float r = rgb[i] - tgt[i];
        acc += fabsf(r);
        dLdC[i] = scale * (float)((r > 0.f) - (r < 0.f));
    }
    float t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t * scale;
}

// Fixed-order final reduction: out = {photometric + planar, photometric,
// planar} from the photometric partials and the planar-term partials the
// projection wrote. Thread t adds entries t, t + 256, ... in float64; the warp
// and CTA trees are fixed, so the result does not vary from run to run.
__global__ void __launch_bounds__(kRedThreads) k_loss_final(const float* __restrict__ photo, int n_photo,
                                                            const float* __restrict__ reg, int n_reg,
                                                            float* __restrict__ out, uint32_t* __restrict__ nonfinite) {
    __shared__ double sa[kRedThreads / 32], sb[kRedThreads / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n_photo; i += kRedThreads) a += photo[i];
    for (int i = threadIdx.x; i < n_reg; i += kRedThreads) b += reg[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        out[0] = (float)(ta + tb);
        out[1] = (float)ta;
        out[2] = (float)tb;
        if (!isfinite(ta + tb)) atomicOr(nonfinite, 1u);   // reported by a later call of the library
    }
}

// One Adam step over a persistent grid; each thread updates groups of 4
// consecutive parameters of one row, with the bias corrections of
// adam_bias_begin / adam_bias_end.
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ P, const float* __restrict__ G,
                                              float* __restrict__ M, float* __restrict__ V, int n, int cap,
                                              AdamArgs a, uint32_t* __restrict__ st, double* __restrict__ pw) {
    __shared__ float sbc[3];
    __shared__ double spw[2];
    if (threadIdx.x == 0) adam_bias_begin(a, st, pw, sbc, spw);
    __syncthreads();
    if (sbc[2] == 0.f) {
        const float ibc1 = sbc[0], ibc2 = sbc[1];   // 1 / (1 - beta^t)
        // a non-finite gradient leaves its parameter and moments as they are (and is reported)
        bool bad = false;
        auto upd = [&](float& p, float g, float& m, float& v, float lr) {
            if (!isfinite(g)) {
                bad = true;
                return;
            }
            adam_update(p, g, m, v, lr, a, ibc1, ibc2);
        };
        // grid-stride over the 14 rows x ceil(n / 4) groups of 4 parameters
        const uint32_t nvec = (uint32_t)(n + 3) / 4u, total = nvec * (uint32_t)kParamRows;
        for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
            const uint32_t row = idx / nvec, j = 4u * (idx - row * nvec);
            const float lr = a.lr[row];
            const size_t k = (size_t)row * cap + j;
            if (j + 3u < (uint32_t)n) {
                float4 p = *reinterpret_cast<float4*>(P + k);
                const float4 g = *reinterpret_cast<const float4*>(G + k);
                float4 m = *reinterpret_cast<float4*>(M + k);
                float4 v = *reinterpret_cast<float4*>(V + k);
                upd(p.x, g.x, m.x, v.x, lr);
                upd(p.y, g.y, m.y, v.y, lr);
                upd(p.z, g.z, m.z, v.z, lr);
                upd(p.w, g.w, m.w, v.w, lr);
                *reinterpret_cast<float4*>(P + k) = p;
                *reinterpret_cast<float4*>(M + k) = m;
                *reinterpret_cast<float4*>(V + k) = v;
            } else {
                for (uint32_t e = 0; e < 4u && j + e < (uint32_t)n; ++e)
                    upd(P[k + e], G[k + e], M[k + e], V[k + e], lr);
            }
        }
        if (bad) atomicOr(st + 10, 1u);
    }
    if (threadIdx.x == 0) adam_bias_end(st, pw, sbc, spw, gridDim.x);
}

// PSNR of an image against a reference: per-CTA float64 partial sums of the
// squared differences (fixed grid, fixed order), then one CTA adds the partials
// in index order and writes 10 log10(1 / max(MSE, 1e-12)).
constexpr int kPsnrBlocks = 256;
__global__ void __launch_bounds__(kRedThreads) k_sqerr(const float* __restrict__ a, const float* __restrict__ b,
                                                       size_t n, double* __restrict__ part) {
    __shared__ double sh[kRedThreads / 32];
    double acc = 0.0;
    const size_t stride = (size_t)gridDim.x * kRedThreads;
    for (size_t i = blockIdx.x * (size_t)kRedThreads + threadIdx.x; i < n; i += stride) {
        const float d = a[i] - b[i];
        acc += (double)(d * d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_psnr_final(const double* __restrict__ part, int n_part, size_t n,
                                                            float* __restrict__ out) {
    __shared__ double sh[kRedThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n_part; i += kRedThreads) acc += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w];
        const double mse = fmax(t / (double)n, 1e-12);
        out[0] = (float)(10.0 * log10(1.0 / mse));
    }
}

}  // namespace

cudaError_t launch_psnr(gs_ctx* c, const float* img, const float* ref, size_t n, float* out, cudaStream_t s) {
    const int grid = (int)std::min<size_t>((n + kRedThreads - 1) / kRedThreads, (size_t)kPsnrBlocks);
    c->launches += 2;
    k_sqerr<<<grid, kRedThreads, 0, s>>>(img, ref, n, c->psnr_part);
    k_psnr_final<<<1, kRedThreads, 0, s>>>(c->psnr_part, grid, n, out);
    return cudaGetLastError();
}

int psnr_scratch_doubles() { return kPsnrBlocks; }

// Planar-term partials of the last projection (view 0's CTAs; none without Gaussians).
static int reg_partials(const gs_ctx* c) { return (c->n + 255) / 256; }

cudaError_t launch_loss(gs_ctx* c, const DevConst& k, const float* rgb, const float* target, float* loss_out,
                        cudaStream_t s) {
    const size_t HW = (size_t)c->width * c->height;
    const size_t total = (size_t)c->n_views * 3 * HW;
    const int nb_img = c->n_partials / 2;
    const float scale = k.lambda_color / (float)(3 * HW);
    c->launches += 2;
    k_l1<<<nb_img, kRedThreads, 0, s>>>(rgb, target, total, scale, c->dLdC, c->partials);
    k_loss_final<<<1, kRedThreads, 0, s>>>(c->partials, nb_img, c->reg_part, reg_partials(c), loss_out, c->dcount + 10);
    return cudaGetLastError();
}

cudaError_t launch_loss_tail(gs_ctx* c, const DevConst& k, const float* photo_partials, int n_photo,
                             float* loss_out, cudaStream_t s) {
    (void)k;
    ++c->launches;
    k_loss_final<<<1, kRedThreads, 0, s>>>(photo_partials, n_photo, c->reg_part, reg_partials(c), loss_out,
                                           c->dcount + 10);
    return cudaGetLastError();
}

AdamArgs adam_args(const gs_ctx* c) {
    AdamArgs a;
    static const int group[kParamRows] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3, 4, 4, 4};
    for (int r = 0; r < kParamRows; ++r) a.lr[r] = c->cfg.lr[group[r]];
    a.b1 = c->cfg.beta1;
    a.b2 = c->cfg.beta2;
    a.eps = c->cfg.eps;
    return a;
}

cudaError_t launch_adam(gs_ctx* c, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    const AdamArgs a = adam_args(c);
    ++c->launches;
    const size_t groups = (size_t)kParamRows * ((c->n + 3) / 4);
    const int grid = (int)std::min<size_t>((groups + 255) / 256, (size_t)c->num_sms * 8);
    k_adam<<<grid, 256, 0, s>>>(c->params, c->grads, c->adam_m, c->adam_v, c->n, c->cap, a, c->dcount, c->adam_pw);
    return cudaGetLastError();
}

cudaError_t launch_copy_T(gs_ctx* c, float* T_out, cudaStream_t s) {
    if (T_out == nullptr) return cudaSuccess;
    return cudaMemcpyAsync(T_out, c->T_final, sizeof(float) * (size_t)c->n_views * c->width * c->height,
                           cudaMemcpyDeviceToDevice, s);
}

}  // namespace gs
