// The learned initialiser: a 3-layer MLP 80 -> 128 -> 128 -> 16 (11 used) with
// GELU, on the tensor cores in BF16 with FP32 accumulation, with hand-written
// forward, backward (MSE against converged Gaussian parameters) and Adam. It
// predicts log-scale (3), quaternion (4), opacity logit (1) and colour (3) of
// a Gaussian inserted at a VO point from the keyframe's 5x5 patch around the
// point, its depth and its camera-frame position.
//
// Every matrix product is one strided GEMM C (+)= A B on tcgen05.mma (bf16
// operands in shared memory, f32 accumulators in TMEM): forward X W^T, input
// gradients dZ W and weight gradients dZ^T X (split over the batch with f32
// atomics). Upstream
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

// ---- the strided GEMM C (+)= A B, A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn] (bf16),
// on the 5th-generation tensor cores (tcgen05, TMEM accumulators) ----
//
// One CTA of 4 warps computes a 128 x NT tile of C. Its K range is walked in
// chunks of 64: all threads gather the A (128 x 64) and B (NT x 64) chunks
// from their strided global layout into shared memory in the canonical
// K-major, non-swizzled UMMA layout (8 x 16-byte core matrices; the core at
// row group g and K group j sits at g * 1024 + j * 128 bytes, so the leading
// (K) byte offset is 128 and the stride (row-group) byte offset 1024), then one
// elected thread issues four tcgen05.mma (M = 128, N = NT, K = 16, BF16 in,
// FP32 accumulate in TMEM) and commits them to an mbarrier that all threads
// wait on before the chunk is restaged. The epilogue reads the accumulator
// with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e. tile rows) and
// stores, accumulates or atomically adds it into C. Every wait is bounded: a
// wait that gives up sets *err, and the CTA still frees its TMEM.
constexpr int kTcM = 128, kTcKC = 64;
constexpr uint32_t kTcWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all >> 4), the fixed version bits 46..48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: D = F32 (bits 4..5), A = B = BF16 (bits 7..9,
// 10..12), both K-major (bits 15, 16 clear), N >> 3 in bits 17..22, M >> 4 in 24..28
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kTcWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Gather one 64-wide K chunk of a (rows x K) operand X(r, k) = X[r * s_r + k * s_k] into the
// canonical layout; zero outside rows < R_valid and k < k_end.
__device__ __forceinline__ void tc_stage(uint8_t* dst, int rows, const bf16* __restrict__ X, long s_r, long s_k,
                                         int r0, int R_valid, int k0, int k_end) {
    const bool kvec = s_k == 1 && (s_r % 8) == 0 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    if (kvec) {
        // one 16-byte core-matrix row (8 consecutive k) per step
        for (int e = threadIdx.x; e < rows * (kTcKC / 8); e += 128) {
            const int r = e / (kTcKC / 8), j = e - r * (kTcKC / 8);
            const int gr = r0 + r, gk = k0 + 8 * j;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < R_valid) {
                if (gk + 8 <= k_end) {
                    v = *reinterpret_cast<const uint4*>(X + (long)gr * s_r + gk);
                } else {
                    bf16 t[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        t[q] = gk + q < k_end ? X[(long)gr * s_r + gk + q] : __float2bfloat16_rn(0.f);
                    v = *reinterpret_cast<const uint4*>(t);
                }
            }
            *reinterpret_cast<uint4*>(dst + (r >> 3) * 1024 + j * 128 + (r & 7) * 16) = v;
        }
    } else {
        // element by element, consecutive threads along the unit-stride dimension
        const bool r_fast = s_r == 1;
        for (int e = threadIdx.x; e < rows * kTcKC; e += 128) {
            int r, k;
            if (r_fast) {
                k = e / rows;
                r = e - k * rows;
            } else {
                r = e / kTcKC;
                k = e - r * kTcKC;
            }
            const int gr = r0 + r, gk = k0 + k;
            const bf16 v = (gr < R_valid && gk < k_end) ? X[(long)gr * s_r + (long)gk * s_k] : __float2bfloat16_rn(0.f);
            *reinterpret_cast<bf16*>(dst + (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) = v;
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(128) k_gemm_tc(const bf16* __restrict__ A, long sam, long sak,
                                                 const bf16* __restrict__ B, long sbk, long sbn,
                                                 float* __restrict__ C, int ldc, int M, int N, int K, int k_split,
                                                 int mode, uint32_t* __restrict__ err) {
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 128, "UMMA N for M = 128");
    constexpr uint32_t kCols = NT <= 32 ? 32u : (NT <= 64 ? 64u : 128u);
    __shared__ __align__(1024) uint8_t sa[kTcM * kTcKC * 2];
    __shared__ __align__(1024) uint8_t sb[NT * kTcKC * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * NT;
    const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t bar = smem_u32(&mbar);
    const uint32_t a_base = smem_u32(sa), b_base = smem_u32(sb);
    constexpr uint32_t idesc = umma_idesc_bf16(kTcM, NT);
    bool ok = true, issued = false;
    uint32_t parity = 0;
    for (int k0 = kb; k0 < ke && ok; k0 += kTcKC) {
        tc_stage(sa, kTcM, A, sam, sak, m0, M, k0, ke);
        tc_stage(sb, NT, B, sbn, sbk, n0, N, k0, ke);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < kTcKC / 16; ++kk) {
                const uint64_t ad = umma_desc(a_base + kk * 256, 128, 1024);
                const uint64_t bd = umma_desc(b_base + kk * 256, 128, 1024);
                const uint32_t acc = (issued || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        issued = true;
        ok = mbar_wait(bar, parity);
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (ok) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n >= N) continue;
                    const float val = issued ? __uint_as_float(v[j]) : 0.f;
                    float* dst = C + (long)m * ldc + n;
                    if (mode == 1) {
                        if (issued) atomicAdd(dst, val);
                    } else if (mode == 2) {
                        *dst += val;
                    } else {
                        *dst = val;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(err, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
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

// Training target of the learned initialiser for Gaussian `first + i` of the
// planar [14][cap] parameters: [log-scale (3), unit quaternion with w >= 0
// (q and -q are the same rotation), opacity logit, colour (3), 0 x 5]. A zero
// quaternion stays zero.
__global__ void k_mlp_targets(const float* __restrict__ P, int cap, int first, int count, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const size_t j = (size_t)first + i;
    const size_t C = (size_t)cap;
    float* o = out + (size_t)i * kOutPad;
    const float w = P[6 * C + j], x = P[7 * C + j], y = P[8 * C + j], z = P[9 * C + j];
    const float nrm = sqrtf(w * w + x * x + y * y + z * z);
    const float inv = nrm > 0.f ? (w < 0.f ? -1.f : 1.f) / nrm : 0.f;
    o[0] = P[3 * C + j];
    o[1] = P[4 * C + j];
    o[2] = P[5 * C + j];
    o[3] = w * inv;
    o[4] = x * inv;
    o[5] = y * inv;
    o[6] = z * inv;
    o[7] = P[10 * C + j];
    o[8] = P[11 * C + j];
    o[9] = P[12 * C + j];
    o[10] = P[13 * C + j];
#pragma unroll
    for (int k = kOut; k < kOutPad; ++k) o[k] = 0.f;
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
    uint32_t* err = nullptr;   // device flag: a tensor-core wait gave up
    uint32_t* herr = nullptr;  // pinned copy of it, refreshed after each forward / backward
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

// C (+)= A B on the tcgen05 tensor cores; split-K (f32 atomics) when `split`.
void gemm(const bf16* A, long sam, long sak, const bf16* B, long sbk, long sbn, float* C, int ldc, int M, int N,
          int K, bool split, cudaStream_t s, uint32_t* err, bool accumulate = false) {
    // these products are small (a few MFLOP): spread them over more CTAs, narrower N tiles
    // for the row-parallel products and K splits of 256 rows for the weight gradients
    int splits = 1, kps = K;
    if (split) {
        splits = std::max(1, std::min(256, K / 256));
        kps = ((K + splits - 1) / splits + kTcKC - 1) / kTcKC * kTcKC;
        splits = (K + kps - 1) / kps;
    }
    const int mode = split ? 1 : (accumulate ? 2 : 0);
    int nt = N <= 16 ? 16 : (N <= 32 ? 32 : (N <= 64 ? 64 : 128));
    const int m_tiles = (M + kTcM - 1) / kTcM;
    while (nt > 32 && m_tiles * ((N + nt - 1) / nt) * splits < 128) nt /= 2;
    dim3 grid((N + nt - 1) / nt, (M + kTcM - 1) / kTcM, splits);
    if (nt == 16)
        k_gemm_tc<16><<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kps, mode, err);
    else if (nt == 32)
        k_gemm_tc<32><<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kps, mode, err);
    else if (nt == 64)
        k_gemm_tc<64><<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kps, mode, err);
    else
        k_gemm_tc<128><<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kps, mode, err);
}

// forward of `rows` feature rows (f32 [rows][80]) into M->y [rows][16]
cudaError_t mlp_forward_rows(gs_mlp* M, const float* feat, int rows, cudaStream_t s) {
    const bf16* W1 = M->wb;
    const bf16* W2 = W1 + kHid * kIn;
    const bf16* W3 = W2 + kHid * kHid;
    k_to_bf16<<<kEwBlocks, kEwThreads, 0, s>>>(feat, M->xb, (long)rows * kIn);
    gemm(M->xb, kIn, 1, W1, 1, kIn, M->z1, kHid, rows, kHid, kIn, false, s, M->err);
    k_bias_gelu<<<kEwBlocks, kEwThreads, 0, s>>>(M->z1, M->p + kOffB1, M->h1, (long)rows * kHid, kHid);
    gemm(M->h1, kHid, 1, W2, 1, kHid, M->z2, kHid, rows, kHid, kHid, false, s, M->err);
    k_bias_gelu<<<kEwBlocks, kEwThreads, 0, s>>>(M->z2, M->p + kOffB2, M->h2, (long)rows * kHid, kHid);
    gemm(M->h2, kHid, 1, W3, 1, kHid, M->y, kOutPad, rows, kOutPad, kHid, false, s, M->err);
    k_bias<<<kEwBlocks, kEwThreads, 0, s>>>(M->y, M->p + kOffB3, (long)rows * kOutPad, kOutPad);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int gs_mlp_targets(gs_ctx* c, int first, int count, float* out_dev, void* stream) {
    if (!c || first < 0 || count < 0 || first > c->n || count > c->n - first || (count > 0 && !out_dev))
        return GS_ERR_ARG;
    if (count == 0) return GS_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return GS_ERR_CUDA;
    ++c->launches;
    k_mlp_targets<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(c->params, c->cap, first, count, out_dev);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

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
    ok = ok && cudaMalloc(&M->err, sizeof(uint32_t)) == cudaSuccess && cudaMemset(M->err, 0, sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&M->herr, sizeof(uint32_t)) == cudaSuccess;
    if (ok) *M->herr = 0u;
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
    void* ps[] = {M->p, M->g, M->m, M->v, M->wb, M->part, M->err};
    for (void* q : ps) cudaFree(q);
    if (M->herr) cudaFreeHost(M->herr);
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
    if (*M->herr != 0u) return GS_ERR_TIMEOUT;   // a tensor-core wait of an earlier call gave up
    if (mlp_rows(M, n) != GS_OK) return GS_ERR_OOM;
    if (mlp_forward_rows(M, feat_dev, n, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemcpyAsync(out_dev, M->y, sizeof(float) * (size_t)n * kOutPad, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    return cudaMemcpyAsync(M->herr, M->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess
               ? GS_OK
               : GS_ERR_CUDA;
}

int gs_mlp_backward(gs_mlp* M, const float* feat_dev, const float* target_dev, int n, float* loss_dev, void* stream) {
    if (!M || n <= 0 || !feat_dev || !target_dev) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (*M->herr != 0u) return GS_ERR_TIMEOUT;   // a tensor-core wait of an earlier call gave up
    if (mlp_rows(M, n) != GS_OK) return GS_ERR_OOM;
    if (mlp_forward_rows(M, feat_dev, n, s) != cudaSuccess) return GS_ERR_CUDA;
    const bf16* W2 = M->wb + kHid * kIn;
    const bf16* W3 = W2 + kHid * kHid;
    cudaMemsetAsync(M->g, 0, sizeof(float) * kParams, s);
    k_mse<<<kEwBlocks, kEwThreads, 0, s>>>(M->y, target_dev, n, M->dy, M->dy_lo, M->g + kOffB3, M->part);
    if (loss_dev) k_sum_partials<<<1, 32, 0, s>>>(M->part, kEwBlocks, loss_dev);
    // Upstream gradients enter the tensor cores as bf16 hi + lo pairs: two products each.
    // output layer: dW3 = dY^T H2, dH2 = dY W3
    for (const bf16* d : {M->dy, M->dy_lo}) gemm(d, 1, kOutPad, M->h2, kHid, 1, M->g + kOffW3, kHid, kOutPad, kHid, n, true, s, M->err);
    gemm(M->dy, kOutPad, 1, W3, kHid, 1, M->dh, kHid, n, kHid, kOutPad, false, s, M->err);
    gemm(M->dy_lo, kOutPad, 1, W3, kHid, 1, M->dh, kHid, n, kHid, kOutPad, false, s, M->err, true);
    k_gelu_back<<<kEwBlocks, kEwThreads, 0, s>>>(M->dh, M->z2, M->dz, M->dz_lo, M->g + kOffB2, n);
    // second layer: dW2 = dZ2^T H1, dH1 = dZ2 W2
    for (const bf16* d : {M->dz, M->dz_lo}) gemm(d, 1, kHid, M->h1, kHid, 1, M->g + kOffW2, kHid, kHid, kHid, n, true, s, M->err);
    gemm(M->dz, kHid, 1, W2, kHid, 1, M->dh, kHid, n, kHid, kHid, false, s, M->err);
    gemm(M->dz_lo, kHid, 1, W2, kHid, 1, M->dh, kHid, n, kHid, kHid, false, s, M->err, true);
    k_gelu_back<<<kEwBlocks, kEwThreads, 0, s>>>(M->dh, M->z1, M->dz, M->dz_lo, M->g + kOffB1, n);
    // first layer: dW1 = dZ1^T X
    for (const bf16* d : {M->dz, M->dz_lo}) gemm(d, 1, kHid, M->xb, kIn, 1, M->g + kOffW1, kIn, kHid, kIn, n, true, s, M->err);
    // the padding rows of the output layer are not trained
    cudaMemsetAsync(M->g + kOffW3 + kOut * kHid, 0, sizeof(float) * (kOutPad - kOut) * kHid, s);
    cudaMemsetAsync(M->g + kOffB3 + kOut, 0, sizeof(float) * (kOutPad - kOut), s);
    cudaMemcpyAsync(M->herr, M->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
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
