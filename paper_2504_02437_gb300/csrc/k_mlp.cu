// The learned initialiser: a 3-layer MLP 80 -> 128 -> 128 -> 16 (11 used) with
// GELU, on the tensor cores in BF16 with FP32 accumulation, with hand-written
// forward, backward (MSE against converged Gaussian parameters) and Adam. It
// predicts log-scale (3), quaternion (4), opacity logit (1) and colour (3) of
// a Gaussian inserted at a VO point from the keyframe's 5x5 patch around the
// point, its depth and its camera-frame position.
//
// Every matrix product is one strided GEMM C (+)= A B on mma.sync m16n8k16
// (bf16 operands, f32 accumulators): forward X W^T, input gradients dZ W and
// weight gradients dZ^T X (split over the batch with f32 atomics). Upstream
// gradients dZ enter as bf16 hi + lo pairs (two products), so the backward
// keeps ~16 mantissa bits where one bf16 rounding would keep 8.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kIn = 80, kHid = 128, kOut = 11, kOutPad = 16;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOutPad * kHid, kParams = kOffB3 + kOutPad;

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M][N] (ldc) = A B (mode 0), += A B with f32 atomics (mode 1, split-K) or
// += A B (mode 2), A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn] (bf16),
// over k in this CTA's split of [0, K). 64 x 64 tile per CTA, 4 warps of 32 x 32
// (2 x 4 mma tiles). Out-of-range elements are staged as zeros.
constexpr int kGT = 64, kGK = 16, kGPad = 8;

__global__ void __launch_bounds__(128) k_gemm_bf16(const bf16* __restrict__ A, long sam, long sak,
                                                   const bf16* __restrict__ B, long sbk, long sbn,
                                                   float* __restrict__ C, int ldc, int M, int N, int K, int k_split,
                                                   int atomic) {
    __shared__ __align__(16) bf16 As[kGT][kGK + kGPad];   // [m][k]
    __shared__ __align__(16) bf16 Bs[kGT][kGK + kGPad];   // [n][k]
    const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
    const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const bf16 zero = __float2bfloat16_rn(0.f);
    for (int k0 = kb; k0 < ke; k0 += kGK) {
        for (int e = threadIdx.x; e < kGT * kGK; e += 128) {
            const int r = e / kGK, kk = e % kGK;
            const int m = m0 + r, n = n0 + r, k = k0 + kk;
            As[r][kk] = (m < M && k < ke) ? A[(long)m * sam + (long)k * sak] : zero;
            Bs[r][kk] = (n < N && k < ke) ? B[(long)k * sbk + (long)n * sbn] : zero;
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + g;
            af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][2 * t]);
            af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * t]);
            af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][2 * t + 8]);
            af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * t + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = wn + 8 * j + g;
            bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * t]);
            bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * t + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + 16 * i + g + (e >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (e & 1);
                if (m < M && n < N) {
                    float* dst = C + (long)m * ldc + n;
                    if (atomic == 1)
                        atomicAdd(dst, acc[i][j][e]);
                    else if (atomic == 2)
                        *dst += acc[i][j][e];
                    else
                        *dst = acc[i][j][e];
                }
            }
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// z <- z + b (kept as the pre-activation), h <- bf16(GELU(z + b)); rows of width `w`
__global__ void k_bias_gelu(float* __restrict__ z, const float* __restrict__ b, bf16* __restrict__ h, long n, int w) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float v = z[i] + b[i % w];
        z[i] = v;
        h[i] = __float2bfloat16_rn(gelu_f(v));
    }
}

__global__ void k_bias(float* __restrict__ y, const float* __restrict__ b, long n, int w) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] += b[i % w];
}

// v = hi + lo with hi = bf16(v), lo = bf16(v - hi): a bf16 pair carrying ~16 mantissa bits
__device__ __forceinline__ void split_bf16(float v, bf16& hi, bf16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// dZ = dH * GELU'(z) as a bf16 hi/lo pair for the next products; the bias gradient sums dZ
// (f32) per column.
__global__ void k_gelu_back(const float* __restrict__ dh, const float* __restrict__ z, bf16* __restrict__ dz,
                            bf16* __restrict__ dz_lo, float* __restrict__ db, int rows) {
    __shared__ float colsum[kHid];
    for (int c = threadIdx.x; c < kHid; c += blockDim.x) colsum[c] = 0.f;
    __syncthreads();
    const long n = (long)rows * kHid;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float v = dh[i] * gelu_grad_f(z[i]);
        split_bf16(v, dz[i], dz_lo[i]);
        atomicAdd(&colsum[i % kHid], v);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kHid; c += blockDim.x) atomicAdd(&db[c], colsum[c]);
}

// MSE over the 11 outputs: dY = 2 (Y - T) / (n 11) (bf16 hi/lo pair, padding columns 0), bias
// gradient of the output layer, and per-block partial loss sums.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ tgt, int rows, bf16* __restrict__ dy,
                      bf16* __restrict__ dy_lo, float* __restrict__ db3, float* __restrict__ partials) {
    __shared__ float colsum[kOutPad];
    __shared__ float red[8];
    for (int c = threadIdx.x; c < kOutPad; c += blockDim.x) colsum[c] = 0.f;
    __syncthreads();
    const float s = 2.f / ((float)rows * (float)kOut);
    float loss = 0.f;
    const long n = (long)rows * kOutPad;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % kOutPad);
        float g = 0.f;
        if (c < kOut) {
            const float r = y[i] - tgt[i];
            loss += r * r;
            g = s * r;
            atomicAdd(&colsum[c], g);
        }
        split_bf16(g, dy[i], dy_lo[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tsum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += red[w];
        partials[blockIdx.x] = tsum / ((float)rows * (float)kOut);
    }
    for (int c = threadIdx.x; c < kOutPad; c += blockDim.x) atomicAdd(&db3[c], colsum[c]);
}

__global__ void k_sum_partials(const float* __restrict__ p, int n, float* __restrict__ out) {
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) a += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if (threadIdx.x == 0) *out = (float)a;
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1,
                           float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_weights_bf16(const float* __restrict__ p, bf16* __restrict__ w) {
    // W1, W2, W3 of the flat layout, contiguous in the bf16 copy
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = kHid * kIn, n2 = kHid * kHid, n3 = kOutPad * kHid;
    if (i < n1) w[i] = __float2bfloat16_rn(p[kOffW1 + i]);
    else if (i < n1 + n2) w[i] = __float2bfloat16_rn(p[kOffW2 + i - n1]);
    else if (i < n1 + n2 + n3) w[i] = __float2bfloat16_rn(p[kOffW3 + i - n1 - n2]);
}

// MLP input of each point: 5x5 RGB patch around its nearest pixel (clamped to the
// image; row-major, RGB interleaved), depth, camera-frame position, 0.
__global__ void k_features(DevCamera cam, const float* __restrict__ image, const float* __restrict__ pts, int n,
                           float* __restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    const float tx = cam.R[0] * x + cam.R[1] * y + cam.R[2] * z + cam.t[0];
    const float ty = cam.R[3] * x + cam.R[4] * y + cam.R[5] * z + cam.t[1];
    const float tz = cam.R[6] * x + cam.R[7] * y + cam.R[8] * z + cam.t[2];
    const float zz = tz > 1e-6f ? tz : 1e-6f;
    const float u = cam.fx * tx / zz + cam.cx, v = cam.fy * ty / zz + cam.cy;
    const int px = (int)fminf(fmaxf(floorf(u + 0.5f), 0.f), (float)(cam.width - 1));
    const int py = (int)fminf(fmaxf(floorf(v + 0.5f), 0.f), (float)(cam.height - 1));
    const size_t HW = (size_t)cam.width * cam.height;
    float* o = f + (size_t)i * kIn;
    int k = 0;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            const int xx = min(max(px + dx, 0), cam.width - 1), yy = min(max(py + dy, 0), cam.height - 1);
            const size_t pix = (size_t)yy * cam.width + xx;
            o[k++] = image[pix];
            o[k++] = image[HW + pix];
            o[k++] = image[2 * HW + pix];
        }
    o[75] = tz;
    o[76] = tx;
    o[77] = ty;
    o[78] = tz;
    o[79] = 0.f;
}

// Gaussian parameters [14][cap] columns base.. of the kept points from the MLP
// outputs [n][16]; a point whose prediction is non-finite or whose log-scale
// leaves [-9, 1] keeps the plain initialisation already staged for it.
__global__ void k_apply_mlp(const float* __restrict__ y, const float* __restrict__ pts, int n,
                            float* __restrict__ stage) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* o = y + (size_t)i * kOutPad;
    bool ok = true;
    for (int c = 0; c < kOut; ++c) ok = ok && isfinite(o[c]);
    for (int c = 0; c < 3; ++c) ok = ok && o[c] >= -9.f && o[c] <= 1.f;
    const float qn = o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6];
    ok = ok && qn > 1e-8f;
    if (!ok) return;
    for (int c = 0; c < 11; ++c) stage[(size_t)(3 + c) * n + i] = o[c];
}

}  // namespace
}  // namespace gs

using namespace gs;

struct gs_mlp {
    int device = 0;
    float* p = nullptr;      // f32 master parameters [kParams]
    float* g = nullptr;      // gradient
    float* m = nullptr;
    float* v = nullptr;
    bf16* wb = nullptr;      // bf16 W1 | W2 | W3
    int t = 0;
    int rows_cap = 0;
    bf16* xb = nullptr;      // [rows][80]
    float* z1 = nullptr;     // [rows][128] pre-activations
    bf16* h1 = nullptr;
    float* z2 = nullptr;
    bf16* h2 = nullptr;
    float* y = nullptr;      // [rows][16]
    bf16* dy = nullptr;
    bf16* dy_lo = nullptr;
    float* dh = nullptr;     // [rows][128] f32 input gradient of a hidden layer
    bf16* dz = nullptr;      // [rows][128] pre-activation gradient, bf16 hi part
    bf16* dz_lo = nullptr;   // ... and lo part
    float* part = nullptr;   // loss partials
};

namespace {

constexpr int kEwBlocks = 256, kEwThreads = 256;

void mlp_free_rows(gs_mlp* M) {
    void* ps[] = {M->xb, M->z1, M->h1, M->z2, M->h2, M->y, M->dy, M->dy_lo, M->dh, M->dz, M->dz_lo};
    for (void* q : ps) cudaFree(q);
    M->xb = nullptr;
    M->z1 = M->z2 = M->y = M->dh = nullptr;
    M->h1 = M->h2 = M->dy = M->dy_lo = M->dz = M->dz_lo = nullptr;
    M->rows_cap = 0;
}

int mlp_rows(gs_mlp* M, int rows) {
    if (rows <= M->rows_cap) return GS_OK;
    mlp_free_rows(M);
    const size_t r = (size_t)std::max(rows, 1024);
    bool ok = cudaMalloc(&M->xb, sizeof(bf16) * r * kIn) == cudaSuccess;
    ok = ok && cudaMalloc(&M->z1, sizeof(float) * r * kHid) == cudaSuccess;
    ok = ok && cudaMalloc(&M->h1, sizeof(bf16) * r * kHid) == cudaSuccess;
    ok = ok && cudaMalloc(&M->z2, sizeof(float) * r * kHid) == cudaSuccess;
    ok = ok && cudaMalloc(&M->h2, sizeof(bf16) * r * kHid) == cudaSuccess;
    ok = ok && cudaMalloc(&M->y, sizeof(float) * r * kOutPad) == cudaSuccess;
    ok = ok && cudaMalloc(&M->dy, sizeof(bf16) * r * kOutPad) == cudaSuccess;
    ok = ok && cudaMalloc(&M->dh, sizeof(float) * r * kHid) == cudaSuccess;
    ok = ok && cudaMalloc(&M->dz, sizeof(bf16) * r * kHid) == cudaSuccess;
    ok = ok && cudaMalloc(&M->dy_lo, sizeof(bf16) * r * kOutPad) == cudaSuccess;
    ok = ok && cudaMalloc(&M->dz_lo, sizeof(bf16) * r * kHid) == cudaSuccess;
    if (!ok) {
        mlp_free_rows(M);
        return GS_ERR_OOM;
    }
    M->rows_cap = (int)r;
    return GS_OK;
}

void gemm(const bf16* A, long sam, long sak, const bf16* B, long sbk, long sbn, float* C, int ldc, int M, int N,
          int K, bool split, cudaStream_t s, bool accumulate = false) {
    int splits = 1, kps = K;
    if (split) {
        splits = std::max(1, std::min(256, K / 1024));
        kps = ((K + splits - 1) / splits + kGK - 1) / kGK * kGK;
        splits = (K + kps - 1) / kps;
    }
    dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT, splits);
    k_gemm_bf16<<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kps, split ? 1 : (accumulate ? 2 : 0));
}

// forward of `rows` feature rows (f32 [rows][80]) into M->y [rows][16]
cudaError_t mlp_forward_rows(gs_mlp* M, const float* feat, int rows, cudaStream_t s) {
    const bf16* W1 = M->wb;
    const bf16* W2 = W1 + kHid * kIn;
    const bf16* W3 = W2 + kHid * kHid;
    k_to_bf16<<<kEwBlocks, kEwThreads, 0, s>>>(feat, M->xb, (long)rows * kIn);
    gemm(M->xb, kIn, 1, W1, 1, kIn, M->z1, kHid, rows, kHid, kIn, false, s);
    k_bias_gelu<<<kEwBlocks, kEwThreads, 0, s>>>(M->z1, M->p + kOffB1, M->h1, (long)rows * kHid, kHid);
    gemm(M->h1, kHid, 1, W2, 1, kHid, M->z2, kHid, rows, kHid, kHid, false, s);
    k_bias_gelu<<<kEwBlocks, kEwThreads, 0, s>>>(M->z2, M->p + kOffB2, M->h2, (long)rows * kHid, kHid);
    gemm(M->h2, kHid, 1, W3, 1, kHid, M->y, kOutPad, rows, kOutPad, kHid, false, s);
    k_bias<<<kEwBlocks, kEwThreads, 0, s>>>(M->y, M->p + kOffB3, (long)rows * kOutPad, kOutPad);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int gs_mlp_create(int device, uint64_t seed, gs_mlp** out) {
    if (!out) return GS_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return GS_ERR_CUDA;
    gs_mlp* M = new gs_mlp();
    M->device = device;
    bool ok = cudaMalloc(&M->p, sizeof(float) * kParams) == cudaSuccess;
    ok = ok && cudaMalloc(&M->g, sizeof(float) * kParams) == cudaSuccess;
    ok = ok && cudaMalloc(&M->m, sizeof(float) * kParams) == cudaSuccess;
    ok = ok && cudaMalloc(&M->v, sizeof(float) * kParams) == cudaSuccess;
    ok = ok && cudaMalloc(&M->wb, sizeof(bf16) * (kHid * kIn + kHid * kHid + kOutPad * kHid)) == cudaSuccess;
    ok = ok && cudaMalloc(&M->part, sizeof(float) * (kEwBlocks + 1)) == cudaSuccess;
    if (!ok) {
        gs_mlp_destroy(M);
        return GS_ERR_OOM;
    }
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from SplitMix64, zero biases; output rows >= 11 zero
    float* h = (float*)calloc(kParams, sizeof(float));
    uint64_t st = seed;
    auto uni = [&st]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int i = 0; i < kHid * kIn; ++i) h[kOffW1 + i] = (float)((2 * uni() - 1) / std::sqrt((double)kIn));
    for (int i = 0; i < kHid * kHid; ++i) h[kOffW2 + i] = (float)((2 * uni() - 1) / std::sqrt((double)kHid));
    for (int i = 0; i < kOut * kHid; ++i) h[kOffW3 + i] = (float)((2 * uni() - 1) / std::sqrt((double)kHid));
    cudaError_t e = cudaMemcpy(M->p, h, sizeof(float) * kParams, cudaMemcpyHostToDevice);
    free(h);
    if (e == cudaSuccess) e = gs_mlp_set_params(M, M->p, nullptr) == GS_OK ? cudaSuccess : cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        gs_mlp_destroy(M);
        return GS_ERR_CUDA;
    }
    *out = M;
    return GS_OK;
}

void gs_mlp_destroy(gs_mlp* M) {
    if (!M) return;
    cudaSetDevice(M->device);
    mlp_free_rows(M);
    void* ps[] = {M->p, M->g, M->m, M->v, M->wb, M->part};
    for (void* q : ps) cudaFree(q);
    delete M;
}

int gs_mlp_set_params(gs_mlp* M, const float* flat_dev, void* stream) {
    if (!M || !flat_dev) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (flat_dev != M->p && cudaMemcpyAsync(M->p, flat_dev, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, s) !=
                                cudaSuccess)
        return GS_ERR_CUDA;
    cudaMemsetAsync(M->m, 0, sizeof(float) * kParams, s);
    cudaMemsetAsync(M->v, 0, sizeof(float) * kParams, s);
    cudaMemsetAsync(M->g, 0, sizeof(float) * kParams, s);
    M->t = 0;
    k_weights_bf16<<<(kHid * kIn + kHid * kHid + kOutPad * kHid + 255) / 256, 256, 0, s>>>(M->p, M->wb);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int gs_mlp_get_params(gs_mlp* M, float* flat_dev, void* stream) {
    if (!M || !flat_dev) return GS_ERR_ARG;
    return cudaMemcpyAsync(flat_dev, M->p, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) ==
                   cudaSuccess
               ? GS_OK
               : GS_ERR_CUDA;
}

int gs_mlp_get_grads(gs_mlp* M, float* flat_dev, void* stream) {
    if (!M || !flat_dev) return GS_ERR_ARG;
    return cudaMemcpyAsync(flat_dev, M->g, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) ==
                   cudaSuccess
               ? GS_OK
               : GS_ERR_CUDA;
}

int gs_mlp_features(const gs_camera* cam, const float* image_dev, const float* points_dev, int n, float* feat_dev,
                    void* stream) {
    if (n < 0 || (n > 0 && (!cam || !image_dev || !points_dev || !feat_dev))) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    if (cam->width <= 0 || cam->height <= 0) return GS_ERR_ARG;
    DevCamera d;
    memset(&d, 0, sizeof(d));
    memcpy(d.R, cam->R, sizeof(d.R));
    memcpy(d.t, cam->t, sizeof(d.t));
    d.fx = cam->fx;
    d.fy = cam->fy;
    d.cx = cam->cx;
    d.cy = cam->cy;
    d.width = cam->width;
    d.height = cam->height;
    k_features<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d, image_dev, points_dev, n, feat_dev);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int gs_mlp_forward(gs_mlp* M, const float* feat_dev, int n, float* out_dev, void* stream) {
    if (!M || n < 0 || (n > 0 && (!feat_dev || !out_dev))) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (mlp_rows(M, n) != GS_OK) return GS_ERR_OOM;
    if (mlp_forward_rows(M, feat_dev, n, s) != cudaSuccess) return GS_ERR_CUDA;
    return cudaMemcpyAsync(out_dev, M->y, sizeof(float) * (size_t)n * kOutPad, cudaMemcpyDeviceToDevice, s) ==
                   cudaSuccess
               ? GS_OK
               : GS_ERR_CUDA;
}

int gs_mlp_backward(gs_mlp* M, const float* feat_dev, const float* target_dev, int n, float* loss_dev, void* stream) {
    if (!M || n <= 0 || !feat_dev || !target_dev) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (mlp_rows(M, n) != GS_OK) return GS_ERR_OOM;
    if (mlp_forward_rows(M, feat_dev, n, s) != cudaSuccess) return GS_ERR_CUDA;
    const bf16* W2 = M->wb + kHid * kIn;
    const bf16* W3 = W2 + kHid * kHid;
    cudaMemsetAsync(M->g, 0, sizeof(float) * kParams, s);
    k_mse<<<kEwBlocks, kEwThreads, 0, s>>>(M->y, target_dev, n, M->dy, M->dy_lo, M->g + kOffB3, M->part);
    if (loss_dev) k_sum_partials<<<1, 32, 0, s>>>(M->part, kEwBlocks, loss_dev);
    // Upstream gradients enter the tensor cores as bf16 hi + lo pairs: two products each.
    // output layer: dW3 = dY^T H2, dH2 = dY W3
    for (const bf16* d : {M->dy, M->dy_lo}) gemm(d, 1, kOutPad, M->h2, kHid, 1, M->g + kOffW3, kHid, kOutPad, kHid, n, true, s);
    gemm(M->dy, kOutPad, 1, W3, kHid, 1, M->dh, kHid, n, kHid, kOutPad, false, s);
    gemm(M->dy_lo, kOutPad, 1, W3, kHid, 1, M->dh, kHid, n, kHid, kOutPad, false, s, true);
    k_gelu_back<<<kEwBlocks, kEwThreads, 0, s>>>(M->dh, M->z2, M->dz, M->dz_lo, M->g + kOffB2, n);
    // second layer: dW2 = dZ2^T H1, dH1 = dZ2 W2
    for (const bf16* d : {M->dz, M->dz_lo}) gemm(d, 1, kHid, M->h1, kHid, 1, M->g + kOffW2, kHid, kHid, kHid, n, true, s);
    gemm(M->dz, kHid, 1, W2, kHid, 1, M->dh, kHid, n, kHid, kHid, false, s);
    gemm(M->dz_lo, kHid, 1, W2, kHid, 1, M->dh, kHid, n, kHid, kHid, false, s, true);
    k_gelu_back<<<kEwBlocks, kEwThreads, 0, s>>>(M->dh, M->z1, M->dz, M->dz_lo, M->g + kOffB1, n);
    // first layer: dW1 = dZ1^T X
    for (const bf16* d : {M->dz, M->dz_lo}) gemm(d, 1, kHid, M->xb, kIn, 1, M->g + kOffW1, kIn, kHid, kIn, n, true, s);
    // the padding rows of the output layer are not trained
    cudaMemsetAsync(M->g + kOffW3 + kOut * kHid, 0, sizeof(float) * (kOutPad - kOut) * kHid, s);
    cudaMemsetAsync(M->g + kOffB3 + kOut, 0, sizeof(float) * (kOutPad - kOut), s);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int gs_mlp_step(gs_mlp* M, float lr, void* stream) {
    if (!M || !(lr > 0.f)) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    M->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, s>>>(M->p, M->g, M->m, M->v, kParams, lr, (float)b1, (float)b2, 1e-8f,
                                                     (float)(1.0 - std::pow(b1, M->t)), (float)(1.0 - std::pow(b2, M->t)));
    k_weights_bf16<<<(kHid * kIn + kHid * kHid + kOutPad * kHid + 255) / 256, 256, 0, s>>>(M->p, M->wb);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int gs_mlp_num_params(void) { return kParams; }

}  // extern "C"

namespace gs {

// Learned initial parameters for the staged points [14][n] (plain values stay where the MLP
// gives none): features -> MLP -> k_apply_mlp.
cudaError_t mlp_initialise(gs_mlp* M, const DevCamera& cam, const float* image, const float* pts, int n, float* stage,
                           float* feat_tmp, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (mlp_rows(M, n) != GS_OK) return cudaErrorMemoryAllocation;
    k_features<<<(n + 127) / 128, 128, 0, s>>>(cam, image, pts, n, feat_tmp);
    cudaError_t e = mlp_forward_rows(M, feat_tmp, n, s);
    if (e != cudaSuccess) return e;
    k_apply_mlp<<<(n + 127) / 128, 128, 0, s>>>(M->y, pts, n, stage);
    return cudaGetLastError();
}

}  // namespace gs
