// The SSIM term of Eq. 10 (Section 3.2 "Map Optimization"):
//   L_color = (1 - lambda_photo) L1 + lambda_photo (1 - SSIM),
// SSIM averaged over the 3HW channel-pixels of a view, with the 3DGS
// lineage's window: an 11 x 11 Gaussian (sigma 1.5) normalised to sum 1,
// zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2.
//
// Forward: per (plane, 32 x 32 tile) CTA, the rendered image x and the
// target y are staged with a 5-pixel halo; the five local moments (mu_x, mu_y,
// E[x^2], E[y^2], E[xy]) are blurred separably (rows, then columns), and each
// pixel q stores SSIM(q) and the three partial derivatives of SSIM(q) with
// respect to mu_x(q), E[x^2](q) and E[xy](q).
// Backward: dSSIM/dx(p) = sum_q w(q - p) [d/dmu_x + 2 x(p) d/dE[x^2]
// + y(p) d/dE[xy]](q): the three derivative maps are blurred the same way
// (the window is symmetric; pixels q outside the image do not exist, so the
// maps are zero-padded), and dL/dC combines it with the L1 sign term.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kSsimTile = 32;
constexpr int kSsimRadius = 5;
constexpr int kSsimSpan = kSsimTile + 2 * kSsimRadius;   // 42
constexpr int kSsimThreads = 256;
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;

struct SsimWindow {
    float w[2 * kSsimRadius + 1];
};

__device__ __forceinline__ float ssim_block_sum(float v, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < kSsimThreads / 32; ++k) t += sh[k];
    return t;   // valid in thread 0
}

// Stage a plane's (kSsimSpan)^2 window around the tile, zero outside the image.
__device__ __forceinline__ void stage_plane(const float* __restrict__ src, int W, int H, int x0, int y0,
                                            float (&dst)[kSsimSpan][kSsimSpan]) {
    for (int i = threadIdx.x; i < kSsimSpan * kSsimSpan; i += kSsimThreads) {
        const int r = i / kSsimSpan, cc = i - r * kSsimSpan;
        const int gx = x0 - kSsimRadius + cc, gy = y0 - kSsimRadius + r;
        dst[r][cc] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? src[(size_t)gy * W + gx] : 0.f;
    }
}

__global__ void __launch_bounds__(kSsimThreads) k_ssim_fwd(const float* __restrict__ x, const float* __restrict__ y,
                                                           const float* const* __restrict__ y_slot, int W, int H, SsimWindow win, float neg_scale,
                                                           float constant, float* __restrict__ d_mu,
                                                           float* __restrict__ d_xx, float* __restrict__ d_xy,
                                                           float* __restrict__ partials) {
    __shared__ float sx[kSsimSpan][kSsimSpan], sy[kSsimSpan][kSsimSpan];
    __shared__ float hb[5][kSsimSpan][kSsimTile];
    __shared__ float red[kSsimThreads / 32];
    if (y_slot != nullptr) y = *y_slot;   // a replayed graph's per-call target
    const int plane = blockIdx.z;
    const size_t HW = (size_t)W * H, off = (size_t)plane * HW;
    const int x0 = blockIdx.x * kSsimTile, y0 = blockIdx.y * kSsimTile;
    stage_plane(x + off, W, H, x0, y0, sx);
    stage_plane(y + off, W, H, x0, y0, sy);
    __syncthreads();
    // rows: blur along x for every staged row
    for (int i = threadIdx.x; i < kSsimSpan * kSsimTile; i += kSsimThreads) {
        const int r = i / kSsimTile, cc = i - r * kSsimTile;
        float a = 0.f, b = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kSsimRadius; ++k) {
            const float wk = win.w[k], u = sx[r][cc + k], v = sy[r][cc + k];
            a = fmaf(wk, u, a);
            b = fmaf(wk, v, b);
            xx = fmaf(wk, u * u, xx);
            yy = fmaf(wk, v * v, yy);
            xy = fmaf(wk, u * v, xy);
        }
        hb[0][r][cc] = a;
        hb[1][r][cc] = b;
        hb[2][r][cc] = xx;
        hb[3][r][cc] = yy;
        hb[4][r][cc] = xy;
    }
    __syncthreads();
    float acc = 0.f;
    for (int i = threadIdx.x; i < kSsimTile * kSsimTile; i += kSsimThreads) {
        const int r = i / kSsimTile, cc = i - r * kSsimTile;
        const int gx = x0 + cc, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k <= 2 * kSsimRadius; ++k) {
            const float wk = win.w[k];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmaf(wk, hb[q][r + k][cc], m[q]);
        }
        const float mx = m[0], my = m[1];
        const float A = 2.f * mx * my + kSsimC1;
        const float B = 2.f * (m[4] - mx * my) + kSsimC2;
        const float Cc = mx * mx + my * my + kSsimC1;
        const float D = (m[2] - mx * mx) + (m[3] - my * my) + kSsimC2;
        const float iden = 1.f / (Cc * D);
        const float s = A * B * iden;
        acc += s;
        // partial derivatives of s with respect to mu_x, E[x^2], E[xy]
        const float g_mu = (2.f * my * (B - A)) * iden - s * (2.f * mx * (D - Cc)) / (Cc * D);
        const float g_xx = -s / D;
        const float g_xy = 2.f * A * iden;
        const size_t o = off + (size_t)gy * W + gx;
        d_mu[o] = g_mu;
        d_xx[o] = g_xx;
        d_xy[o] = g_xy;
    }
    const float t = ssim_block_sum(acc, red);
    if (threadIdx.x == 0) {
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[bid] = t * neg_scale + (bid == 0 ? constant : 0.f);
    }
}

__global__ void __launch_bounds__(kSsimThreads) k_ssim_bwd(const float* __restrict__ x, const float* __restrict__ y,
                                                           const float* const* __restrict__ y_slot, int W, int H,
                                                           SsimWindow win,
                                                           const float* __restrict__ d_mu,
                                                           const float* __restrict__ d_xx,
                                                           const float* __restrict__ d_xy, float l1_scale,
                                                           float ssim_scale, float* __restrict__ dLdC,
                                                           float* __restrict__ partials) {
    __shared__ float sg[3][kSsimSpan][kSsimSpan];
    __shared__ float hb[3][kSsimSpan][kSsimTile];
    __shared__ float red[kSsimThreads / 32];
    if (y_slot != nullptr) y = *y_slot;
    const int plane = blockIdx.z;
    const size_t HW = (size_t)W * H, off = (size_t)plane * HW;
    const int x0 = blockIdx.x * kSsimTile, y0 = blockIdx.y * kSsimTile;
    stage_plane(d_mu + off, W, H, x0, y0, sg[0]);
    stage_plane(d_xx + off, W, H, x0, y0, sg[1]);
    stage_plane(d_xy + off, W, H, x0, y0, sg[2]);
    __syncthreads();
    for (int i = threadIdx.x; i < kSsimSpan * kSsimTile; i += kSsimThreads) {
        const int r = i / kSsimTile, cc = i - r * kSsimTile;
        float a = 0.f, b = 0.f, e = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kSsimRadius; ++k) {
            const float wk = win.w[k];
            a = fmaf(wk, sg[0][r][cc + k], a);
            b = fmaf(wk, sg[1][r][cc + k], b);
            e = fmaf(wk, sg[2][r][cc + k], e);
        }
        hb[0][r][cc] = a;
        hb[1][r][cc] = b;
        hb[2][r][cc] = e;
    }
    __syncthreads();
    float acc = 0.f;
    for (int i = threadIdx.x; i < kSsimTile * kSsimTile; i += kSsimThreads) {
        const int r = i / kSsimTile, cc = i - r * kSsimTile;
        const int gx = x0 + cc, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        float a = 0.f, b = 0.f, e = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kSsimRadius; ++k) {
            const float wk = win.w[k];
            a = fmaf(wk, hb[0][r + k][cc], a);
            b = fmaf(wk, hb[1][r + k][cc], b);
            e = fmaf(wk, hb[2][r + k][cc], e);
        }
        const size_t o = off + (size_t)gy * W + gx;
        const float xp = x[o], yp = y[o];
        const float dS = a + 2.f * xp * b + yp * e;
        const float res = xp - yp;
        acc += fabsf(res);
        dLdC[o] = l1_scale * (float)((res > 0.f) - (res < 0.f)) - ssim_scale * dS;
    }
    const float t = ssim_block_sum(acc, red);
    if (threadIdx.x == 0) partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t * l1_scale;
}

SsimWindow make_window() {
    SsimWindow win;
    double g[2 * kSsimRadius + 1], s = 0.0;
    for (int k = 0; k <= 2 * kSsimRadius; ++k) {
        const double d = k - kSsimRadius;
        g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k <= 2 * kSsimRadius; ++k) win.w[k] = (float)(g[k] / s);
    return win;
}

}  // namespace

int ssim_blocks(int width, int height, int n_views) {
    return n_views * 3 * ((width + kSsimTile - 1) / kSsimTile) * ((height + kSsimTile - 1) / kSsimTile);
}

// L_color with the SSIM term for the rendered views: writes dL/dC and, into
// `partials` (2 ssim_blocks entries), the photometric loss as per-CTA terms.
cudaError_t launch_ssim_loss(gs_ctx* c, const DevConst& k, const float* rgb, const float* target,
                             const float* const* target_slot, float* partials, cudaStream_t s) {
    const int W = c->width, H = c->height, V = c->n_views;
    const float lp = c->cfg.lambda_photo;
    const float inv = 1.f / (float)(3 * (size_t)W * H);
    const float l1_scale = k.lambda_color * (1.f - lp) * inv, ssim_scale = k.lambda_color * lp * inv;
    const size_t HW = (size_t)W * H * 3 * V;
    float *d_mu = c->ssim_maps, *d_xx = c->ssim_maps + HW, *d_xy = c->ssim_maps + 2 * HW;
    const dim3 grid((W + kSsimTile - 1) / kSsimTile, (H + kSsimTile - 1) / kSsimTile, 3 * V);
    const int nb = ssim_blocks(W, H, V);
    const SsimWindow win = make_window();
    c->launches += 2;
    k_ssim_fwd<<<grid, kSsimThreads, 0, s>>>(rgb, target, target_slot, W, H, win, -ssim_scale, k.lambda_color * lp * (float)V,
                                             d_mu, d_xx, d_xy, partials);
    k_ssim_bwd<<<grid, kSsimThreads, 0, s>>>(rgb, target, target_slot, W, H, win, d_mu, d_xx, d_xy, l1_scale, ssim_scale,
                                             c->dLdC, partials + nb);
    return cudaGetLastError();
}

}  // namespace gs
