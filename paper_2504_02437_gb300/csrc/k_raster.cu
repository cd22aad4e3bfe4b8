// Front-to-back alpha compositing (Eq. 3, Section 3.1) and its adjoint.
//
// One CTA per (view, tile); one thread per pixel. Each warp owns an 8x4 pixel
// block so that a Gaussian that misses the whole block can be skipped by the
// warp. The tile's sorted pair list is walked in batches of one record per
// thread staged in shared memory (gathered by Gaussian id from the 48-byte
// raster records).
//
// Membership is pixel-exact (|px - u| <= r and |py - v| <= r), so the image is
// the same for every tile size: tiles only bound which Gaussians a pixel tests.
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exponent of the Gaussian in base 2, written with explicit rounding so that the
// forward and backward kernels take bit-identical alpha decisions
__device__ __forceinline__ float power2(const float4 q, float dx, float dy) {
    float t = __fmul_rn(__fmul_rn(q.z, dy), dy);
    t = __fmaf_rn(__fmul_rn(q.y, dx), dy, t);
    return __fmaf_rn(__fmul_rn(q.x, dx), dx, t);
}

// Stage one raster record relative to the local origin (ox, oy), the tile's
// corner rounded down to a multiple of 32 px. The screen mean is stored split
// (integer part in f0.xy, fractions in f1.w, f2.w); the local mean
// (ui - ox) + uf is formed once per pair and tile, so pixel offsets carry the
// rounding of a small number only, and the same for tiles of 8, 16 or 32 px
// (which keeps the image bit-identical across tile sizes).
__device__ __forceinline__ void load_record(const float4* __restrict__ rec, uint32_t item, float ox, float oy,
                                            float4& s0, float4& s1, float4& s2) {
    const float4 a = rec[(size_t)item * 3 + 0];
    const float4 q = rec[(size_t)item * 3 + 1];
    const float4 c = rec[(size_t)item * 3 + 2];
    s0 = make_float4((a.x - ox) + q.w, (a.y - oy) + c.w, a.z, a.w);
    s1 = q;
    s2 = c;
}

// pixel of thread `tid` inside a TILE x TILE tile: warps cover 8x4 blocks
template <int TILE>
__device__ __forceinline__ void pixel_of(int tid, int& lx, int& ly) {
    constexpr int BX = TILE / 8;     // 8-wide blocks per tile row
    int w = tid >> 5, l = tid & 31;
    lx = (w % BX) * 8 + (l & 7);
    ly = (w / BX) * 4 + (l >> 3);
}

template <int TILE>
__global__ void __launch_bounds__(TILE* TILE) k_raster_fwd(const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ pval,
                                                           const float4* __restrict__ rec, int width, int height,
                                                           int tiles_x, int tiles_per_view, int n, DevConst kc,
                                                           float* __restrict__ out_rgb, float* __restrict__ out_T,
                                                           uint32_t* __restrict__ out_last,
                                                           int32_t* __restrict__ out_argmax) {
    constexpr int BLOCK = TILE * TILE;
    __shared__ float4 s0[BLOCK], s1[BLOCK], s2[BLOCK];
    __shared__ uint32_t sid[BLOCK];
    const int bin = blockIdx.x;
    const int view = bin / tiles_per_view;
    const int t = bin - view * tiles_per_view;
    const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
    int lx, ly;
    pixel_of<TILE>(threadIdx.x, lx, ly);
    const int px = txi * TILE + lx, py = tyi * TILE + ly;
    const bool inside = px < width && py < height;
    // pixel offsets are taken from a 32-px-aligned local origin (see load_record)
    const float ox = (float)((txi * TILE) & ~31), oy = (float)((tyi * TILE) & ~31);
    const float fx = (float)px - ox, fy = (float)py - oy;
    const uint2 rg = ranges[bin];
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    uint32_t last = 0;
    float wmax = -1.f;
    uint32_t amax = 0xFFFFFFFFu;
    bool done = !inside;
    for (uint32_t bs = rg.x; bs < rg.y; bs += BLOCK) {
        if (__syncthreads_count(done) == BLOCK) break;
        uint32_t j = bs + threadIdx.x;
        if (j < rg.y) {
            uint32_t item = pval[j];
            load_record(rec, item, ox, oy, s0[threadIdx.x], s1[threadIdx.x], s2[threadIdx.x]);
            sid[threadIdx.x] = item;
        }
        __syncthreads();
        const int cnt = min((uint32_t)BLOCK, rg.y - bs);
        for (int k = 0; k < cnt && !done; ++k) {
            const float4 a = s0[k];
            const float dx = fx - a.x, dy = fy - a.y;
            if (fabsf(dx) > a.z || fabsf(dy) > a.z) continue;
            const float4 q = s1[k];
            const float alpha = fminf(kc.alpha_max, __fmul_rn(a.w, ex2_approx(power2(q, dx, dy))));
            if (alpha < kc.alpha_min) continue;
            const float Tn = __fmul_rn(T, 1.f - alpha);
            if (Tn < kc.T_min) {
                done = true;
                break;
            }
            const float wgt = alpha * T;
            const float4 c = s2[k];
            cr = fmaf(c.x, wgt, cr);
            cg = fmaf(c.y, wgt, cg);
            cb = fmaf(c.z, wgt, cb);
            T = Tn;
            last = bs + k - rg.x + 1;
            if (out_argmax != nullptr && wgt > wmax) {
                wmax = wgt;
                amax = sid[k];
            }
        }
    }
    if (inside) {
        const size_t HW = (size_t)width * height;
        const size_t pix = (size_t)py * width + px;
        out_rgb[(size_t)view * 3 * HW + pix] = cr;
        out_rgb[(size_t)view * 3 * HW + HW + pix] = cg;
        out_rgb[(size_t)view * 3 * HW + 2 * HW + pix] = cb;
        out_T[view * HW + pix] = T;
        out_last[view * HW + pix] = last;
        if (out_argmax != nullptr)
            out_argmax[view * HW + pix] = amax == 0xFFFFFFFFu ? -1 : (int32_t)(amax - (uint32_t)view * n);
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

template <int TILE>
__global__ void __launch_bounds__(TILE* TILE) k_raster_bwd(const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ pval,
                                                           const float4* __restrict__ rec, int width, int height,
                                                           int tiles_x, int tiles_per_view, DevConst kc,
                                                           const float* __restrict__ T_final,
                                                           const uint32_t* __restrict__ n_last,
                                                           const float* __restrict__ dLdC,
                                                           float* __restrict__ grad2d) {
    constexpr int BLOCK = TILE * TILE;
    __shared__ float4 s0[BLOCK], s1[BLOCK], s2[BLOCK];
    __shared__ uint32_t sid[BLOCK];
    __shared__ uint32_t smax;
    const int bin = blockIdx.x;
    const int view = bin / tiles_per_view;
    const int t = bin - view * tiles_per_view;
    const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
    int lx, ly;
    pixel_of<TILE>(threadIdx.x, lx, ly);
    const int px = txi * TILE + lx, py = tyi * TILE + ly;
    const bool inside = px < width && py < height;
    const float ox = (float)((txi * TILE) & ~31), oy = (float)((tyi * TILE) & ~31);
    const float fx = (float)px - ox, fy = (float)py - oy;
    const uint2 rg = ranges[bin];
    const size_t HW = (size_t)width * height;
    const size_t pix = (size_t)py * width + px;
    float T = 1.f, gr = 0.f, gg = 0.f, gb = 0.f;
    uint32_t mine = 0;
    if (inside) {
        T = T_final[view * HW + pix];
        mine = n_last[view * HW + pix];
        gr = dLdC[(size_t)view * 3 * HW + pix];
        gg = dLdC[(size_t)view * 3 * HW + HW + pix];
        gb = dLdC[(size_t)view * 3 * HW + 2 * HW + pix];
    }
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    uint32_t wm = __reduce_max_sync(0xFFFFFFFFu, mine);
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, wm);
    __syncthreads();
    const uint32_t end = rg.x + smax;
    const uint32_t my_end = rg.x + mine;     // entries at positions < my_end may blend
    float ar = 0.f, ag = 0.f, ab = 0.f;      // colour accumulated behind, normalised by T
    for (uint32_t be = end; be > rg.x;) {
        const uint32_t bs = be > rg.x + BLOCK ? be - BLOCK : rg.x;
        __syncthreads();
        uint32_t j = bs + threadIdx.x;
        if (j < be) {
            uint32_t item = pval[j];
            load_record(rec, item, ox, oy, s0[threadIdx.x], s1[threadIdx.x], s2[threadIdx.x]);
            sid[threadIdx.x] = item;
        }
        __syncthreads();
        for (int k = (int)(be - bs) - 1; k >= 0; --k) {
            const uint32_t pos = bs + k;
            const float4 a = s0[k];
            const float dx = fx - a.x, dy = fy - a.y;
            bool contrib = pos < my_end && fabsf(dx) <= a.z && fabsf(dy) <= a.z;
            const float4 q = s1[k];
            const float G = ex2_approx(power2(q, dx, dy));
            const float oG = __fmul_rn(a.w, G);
            const float alpha = fminf(kc.alpha_max, oG);
            contrib = contrib && alpha >= kc.alpha_min;
            if (!__any_sync(0xFFFFFFFFu, contrib)) continue;
            float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_o = 0.f, g_r = 0.f, g_g = 0.f, g_bb = 0.f;
            if (contrib) {
                const float4 c = s2[k];
                const float oma = 1.f - alpha;
                T = T / oma;                             // transmittance in front of this Gaussian
                const float wgt = alpha * T;
                g_r = gr * wgt;
                g_g = gg * wgt;
                g_bb = gb * wgt;
                const float dalpha = T * (gr * (c.x - ar) + gg * (c.y - ag) + gb * (c.z - ab));
                ar = fmaf(alpha, c.x - ar, ar);
                ag = fmaf(alpha, c.y - ag, ag);
                ab = fmaf(alpha, c.z - ab, ab);
                if (oG <= kc.alpha_max) {
                    // dL/dp2 with alpha = o 2^p2
                    const float g2 = dalpha * oG * kLn2;
                    g_u = -g2 * (2.f * q.x * dx + q.y * dy);
                    g_v = -g2 * (q.y * dx + 2.f * q.z * dy);
                    g_a = g2 * dx * dx;
                    g_b = g2 * dx * dy;
                    g_c = g2 * dy * dy;
                    g_o = dalpha * G;
                }
            }
            g_u = warp_sum(g_u);
            g_v = warp_sum(g_v);
            g_a = warp_sum(g_a);
            g_b = warp_sum(g_b);
            g_c = warp_sum(g_c);
            g_o = warp_sum(g_o);
            g_r = warp_sum(g_r);
            g_g = warp_sum(g_g);
            g_bb = warp_sum(g_bb);
            if ((threadIdx.x & 31) == 0) {
                float* dst = grad2d + (size_t)sid[k] * kGrad2dStride;
                atomicAdd(reinterpret_cast<float4*>(dst), make_float4(g_u, g_v, g_a, g_b));
                atomicAdd(reinterpret_cast<float4*>(dst + 4), make_float4(g_c, g_o, g_r, g_g));
                atomicAdd(dst + 8, g_bb);
            }
        }
        be = bs;
    }
}

// Algorithmic work of the last render, by replaying the forward traversal per
// pixel: out[0] += pairs tested by the forward pass (up to and including the
// stopping one), out[1] += pairs blended, out[2] += pairs the backward pass
// walks (entries up to the last blended one).
template <int TILE>
__global__ void __launch_bounds__(TILE* TILE) k_count_work(const uint2* __restrict__ ranges,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ pval, int width, int height,
                                                           int tiles_x, int tiles_per_view, DevConst kc,
                                                           unsigned long long* __restrict__ out) {
    const int bin = blockIdx.x;
    const int view = bin / tiles_per_view;
    const int t = bin - view * tiles_per_view;
    const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
    int lx, ly;
    pixel_of<TILE>(threadIdx.x, lx, ly);
    const int px = txi * TILE + lx, py = tyi * TILE + ly;
    if (px >= width || py >= height) return;
    const float ox = (float)((txi * TILE) & ~31), oy = (float)((tyi * TILE) & ~31);
    const float fx = (float)px - ox, fy = (float)py - oy;
    const uint2 rg = ranges[bin];
    float T = 1.f;
    unsigned long long tested = 0, blended = 0, walked = 0;
    for (uint32_t j = rg.x; j < rg.y; ++j) {
        const uint32_t item = pval[j];
        float4 a, q, c;
        load_record(rec, item, ox, oy, a, q, c);
        ++tested;
        const float dx = fx - a.x, dy = fy - a.y;
        if (fabsf(dx) > a.z || fabsf(dy) > a.z) continue;
        const float alpha = fminf(kc.alpha_max, __fmul_rn(a.w, ex2_approx(power2(q, dx, dy))));
        if (alpha < kc.alpha_min) continue;
        const float Tn = __fmul_rn(T, 1.f - alpha);
        if (Tn < kc.T_min) break;
        T = Tn;
        ++blended;
        walked = j - rg.x + 1;
    }
    atomicAdd(out + 0, tested);
    atomicAdd(out + 1, blended);
    atomicAdd(out + 2, walked);
}

}  // namespace

cudaError_t launch_count_work(gs_ctx* c, const DevConst& k, unsigned long long* out, cudaStream_t s) {
    const int tpv = c->hcam[0].tiles_x * c->hcam[0].tiles_y;
    if (c->n_bins == 0) return cudaSuccess;
    ++c->launches;
    if (c->tile == 16)
        k_count_work<16><<<c->n_bins, 256, 0, s>>>(c->ranges, c->rec, c->pval[c->pair_buf], c->width, c->height,
                                                   c->hcam[0].tiles_x, tpv, k, out);
    else
        k_count_work<8><<<c->n_bins, 64, 0, s>>>(c->ranges, c->rec, c->pval[c->pair_buf], c->width, c->height,
                                                 c->hcam[0].tiles_x, tpv, k, out);
    return cudaGetLastError();
}

cudaError_t launch_raster_forward(gs_ctx* c, const DevConst& k, float* rgb, int32_t* argmax, cudaStream_t s) {
    const int tpv = c->hcam[0].tiles_x * c->hcam[0].tiles_y;
    if (c->n_bins == 0) return cudaSuccess;
    ++c->launches;
    if (c->tile == 16)
        k_raster_fwd<16><<<c->n_bins, 256, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                   c->hcam[0].tiles_x, tpv, c->n, k, rgb, c->T_final, c->n_last,
                                                   argmax);
    else
        k_raster_fwd<8><<<c->n_bins, 64, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                 c->hcam[0].tiles_x, tpv, c->n, k, rgb, c->T_final, c->n_last,
                                                 argmax);
    return cudaGetLastError();
}

cudaError_t launch_raster_backward(gs_ctx* c, const DevConst& k, const float* dLdC, cudaStream_t s) {
    const int tpv = c->hcam[0].tiles_x * c->hcam[0].tiles_y;
    if (c->n_bins == 0) return cudaSuccess;
    ++c->launches;
    if (c->tile == 16)
        k_raster_bwd<16><<<c->n_bins, 256, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                   c->hcam[0].tiles_x, tpv, k, c->T_final, c->n_last, dLdC,
                                                   c->grad2d);
    else
        k_raster_bwd<8><<<c->n_bins, 64, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                 c->hcam[0].tiles_x, tpv, k, c->T_final, c->n_last, dLdC,
                                                 c->grad2d);
    return cudaGetLastError();
}

}  // namespace gs
