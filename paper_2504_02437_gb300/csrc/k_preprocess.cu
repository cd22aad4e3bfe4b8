// Per-Gaussian projection (Eq. 1-2, Section 3.1) and its adjoint.
//
// One thread per (view, Gaussian). Parameters are read from the planar SoA
// [14][cap] (each row coalesced across a warp); outputs are a 48-byte raster
// record per (view, Gaussian), the depth key for the sort, and the number of
// tiles the pixel box touches.
#include "gs_internal.cuh"

namespace gs {
namespace {

// View-independent shape of one Gaussian (Eq. 1): scales, normalised
// quaternion, its rotation and Sigma = R S S^T R^T.
struct Shape {
    float s[3];
    float qn[4];
    float qnorm;
    float R[9];            // row-major
    float S[6];            // Sigma (xx, xy, xz, yy, yz, zz)
};

// View-dependent projection (Eq. 2) of one Gaussian for one camera.
struct Proj {
    float tx, ty, tz;
    float xr, yr;          // x/z, y/z before clamping
    float xh, yh;          // clamped
    float J00, J02, J11, J12;
    float T0[3], T1[3];    // rows of J W
    float A, B, C, det;    // dilated 2D covariance
};

// Float-float ("double-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2, about 48 significant bits. Error-free transformations: TwoSum
// (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct through a fused multiply-add
// (Dekker 1971; with FMA as in Ogita, Rump and Oishi 2005). The intrinsics
// keep the compiler from contracting or reassociating the steps.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ FF quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// r0 m0 + r1 m1 + r2 m2 + t of float32 inputs
__device__ __forceinline__ FF ff_dot3_add(float r0, float m0, float r1, float m1, float r2, float m2, float t) {
    FF acc = two_prod(r0, m0);
    acc = ff_add(acc, two_prod(r1, m1));
    acc = ff_add(acc, two_prod(r2, m2));
    return ff_add(acc, FF{t, 0.f});
}
__device__ __forceinline__ FF ff_div(FF a, FF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const FF p = two_prod(q1, b.hi);
    // remainder a - q1 b, to first order
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), __fsub_rn(a.lo, __fmul_rn(q1, b.lo)));
    return quick_two_sum(q1, __fdiv_rn(r, b.hi));
}
// f a + c
__device__ __forceinline__ FF ff_scale_add(FF a, float f, float c) {
    FF p = two_prod(a.hi, f);
    p = quick_two_sum(p.hi, __fmaf_rn(a.lo, f, p.lo));
    return ff_add(p, FF{c, 0.f});
}
// floor and fraction of hi + lo: returns the integer part, writes the fraction in [0, 1)
__device__ __forceinline__ float ff_floor_frac(FF a, float& frac) {
    float fl = floorf(a.hi);
    float f = __fadd_rn(__fsub_rn(a.hi, fl), a.lo);   // a.hi - fl is exact
    if (f < 0.f) {
        fl -= 1.f;
        f = __fadd_rn(f, 1.f);
    } else if (f >= 1.f) {
        fl += 1.f;
        f = __fsub_rn(f, 1.f);
    }
    frac = fminf(fmaxf(f, 0.f), 0x1.fffffep-1f);
    return fl;
}

__device__ __forceinline__ void load_params(const float* __restrict__ P, int cap, int i, float p[kParamRows]) {
#pragma unroll
    for (int r = 0; r < kParamRows; ++r) p[r] = __ldg(P + (size_t)r * cap + i);
}

// Eq. 1 in float32.
__device__ __forceinline__ void shape_of(const float p[kParamRows], Shape& g) {
    g.s[0] = expf(p[3]);
    g.s[1] = expf(p[4]);
    g.s[2] = expf(p[5]);
    float qq = p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9];
    g.qnorm = sqrtf(qq);
    float inv = 1.0f / g.qnorm;
    float w = p[6] * inv, x = p[7] * inv, y = p[8] * inv, z = p[9] * inv;
    g.qn[0] = w; g.qn[1] = x; g.qn[2] = y; g.qn[3] = z;
    g.R[0] = 1.f - 2.f * (y * y + z * z); g.R[1] = 2.f * (x * y - w * z);       g.R[2] = 2.f * (x * z + w * y);
    g.R[3] = 2.f * (x * y + w * z);       g.R[4] = 1.f - 2.f * (x * x + z * z); g.R[5] = 2.f * (y * z - w * x);
    g.R[6] = 2.f * (x * z - w * y);       g.R[7] = 2.f * (y * z + w * x);       g.R[8] = 1.f - 2.f * (x * x + y * y);
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[i * 3 + k] = g.R[i * 3 + k] * g.s[k];
    g.S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    g.S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    g.S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    g.S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    g.S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    g.S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

// Eq. 2 in float32 for one camera: J at the clamped x/z, y/z; T = J W;
// Sigma2D = T Sigma T^T + dilation I.
__device__ __forceinline__ void project_one(const float p[kParamRows], const Shape& g, const DevCamera& cam,
                                            float dilation, Proj& o) {
    o.tx = cam.R[0] * p[0] + cam.R[1] * p[1] + cam.R[2] * p[2] + cam.t[0];
    o.ty = cam.R[3] * p[0] + cam.R[4] * p[1] + cam.R[5] * p[2] + cam.t[1];
    o.tz = cam.R[6] * p[0] + cam.R[7] * p[1] + cam.R[8] * p[2] + cam.t[2];
    float iz = 1.0f / o.tz;
    o.xr = o.tx * iz;
    o.yr = o.ty * iz;
    o.xh = fminf(fmaxf(o.xr, -cam.lim_x), cam.lim_x);
    o.yh = fminf(fmaxf(o.yr, -cam.lim_y), cam.lim_y);
    o.J00 = cam.fx * iz;
    o.J02 = -cam.fx * o.xh * iz;
    o.J11 = cam.fy * iz;
    o.J12 = -cam.fy * o.yh * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.T0[k] = o.J00 * cam.R[k] + o.J02 * cam.R[6 + k];
        o.T1[k] = o.J11 * cam.R[3 + k] + o.J12 * cam.R[6 + k];
    }
    float ST0[3], ST1[3];
    ST0[0] = g.S[0] * o.T0[0] + g.S[1] * o.T0[1] + g.S[2] * o.T0[2];
    ST0[1] = g.S[1] * o.T0[0] + g.S[3] * o.T0[1] + g.S[4] * o.T0[2];
    ST0[2] = g.S[2] * o.T0[0] + g.S[4] * o.T0[1] + g.S[5] * o.T0[2];
    ST1[0] = g.S[0] * o.T1[0] + g.S[1] * o.T1[1] + g.S[2] * o.T1[2];
    ST1[1] = g.S[1] * o.T1[0] + g.S[3] * o.T1[1] + g.S[4] * o.T1[2];
    ST1[2] = g.S[2] * o.T1[0] + g.S[4] * o.T1[1] + g.S[5] * o.T1[2];
    o.A = o.T0[0] * ST0[0] + o.T0[1] * ST0[1] + o.T0[2] * ST0[2] + dilation;
    o.B = o.T0[0] * ST1[0] + o.T0[1] * ST1[1] + o.T0[2] * ST1[2];
    o.C = o.T1[0] * ST1[0] + o.T1[1] * ST1[1] + o.T1[2] * ST1[2] + dilation;
    o.det = o.A * o.C - o.B * o.B;
}

// Projection of one (view, Gaussian) item; returns whether it is visible (has tiles).
__device__ __forceinline__ bool preprocess_one(const float* __restrict__ P, int n, int cap, int gid, int view,
                                               const DevCamera* __restrict__ cams, const DevConst& kc, int tile,
                                               float4* __restrict__ rec, uint32_t* __restrict__ tiles,
                                               uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval,
                                               float* __restrict__ depth, float& planar) {
    const DevCamera& cam = cams[view];
    size_t item = (size_t)view * n + gid;
    float p[kParamRows];
    load_params(P, cap, gid, p);
    Shape g;
    shape_of(p, g);
    // the Gaussian's planar term of Eq. 10: max(floor, smallest scale)
    planar = fmaxf(kc.reg_floor, fminf(g.s[0], fminf(g.s[1], g.s[2])));
    Proj o;
    project_one(p, g, cam, kc.dilation, o);
    // Screen mean and depth in float-float (the covariance stays float32): the
    // compositing subtracts u from pixel coordinates, and the rounding of u in
    // float32 (about 1e-4 px at 1000 px) would dominate the error of the
    // cancelling sums of the mean gradient.
    const FF tzf = ff_dot3_add(cam.R[6], p[0], cam.R[7], p[1], cam.R[8], p[2], cam.t[2]);
    const FF txf = ff_dot3_add(cam.R[0], p[0], cam.R[1], p[1], cam.R[2], p[2], cam.t[0]);
    const FF tyf = ff_dot3_add(cam.R[3], p[0], cam.R[4], p[1], cam.R[5], p[2], cam.t[1]);
    const float tz32 = tzf.hi;
    bool valid = (tzf.hi > kc.near_z || (tzf.hi == kc.near_z && tzf.lo > 0.f)) && (o.det > 0.f);
    const FF izx = ff_div(txf, tzf), izy = ff_div(tyf, tzf);
    const FF uf2 = ff_scale_add(izx, cam.fx, cam.cx), vf2 = ff_scale_add(izy, cam.fy, cam.cy);
    float idet = 1.0f / o.det;
    float ca = o.C * idet, cb = -o.B * idet, cc = o.A * idet;
    float mid = 0.5f * (o.A + o.C);
    float lam = mid + sqrtf(fmaxf(kc.lambda_floor, mid * mid - o.det));
    float r = ceilf(kc.radius_sigma * sqrtf(lam));
    // screen positions beyond +-2^23 px or radii beyond 2^22 px are culled
    valid = valid && fabsf(uf2.hi) < 8388608.f && fabsf(vf2.hi) < 8388608.f && r < 4194304.f;
    float ui = 0.f, uf = 0.f, vi = 0.f, vf = 0.f;
    uint32_t ntiles = 0;
    if (valid) {
        ui = ff_floor_frac(uf2, uf);
        vi = ff_floor_frac(vf2, vf);
        int x0, x1, y0, y1;
        if (pixel_box(ui, uf, vi, vf, r, cam.width, cam.height, x0, x1, y0, y1))
            ntiles = (uint32_t)((x1 / tile - x0 / tile + 1) * (y1 / tile - y0 / tile + 1));
        else
            valid = false;
    }
    float o_act = 1.0f / (1.0f + expf(-p[10]));
    // conic pre-scaled for exp2: power * log2(e) = a' dx^2 + b' dx dy + c' dy^2
    const float k1 = -0.5f * kLog2e, k2 = -kLog2e;
    rec[item * 3 + 0] = make_float4(ui, vi, valid ? r : -1.f, o_act);
    rec[item * 3 + 1] = make_float4(ca * k1, cb * k2, cc * k1, uf);
    rec[item * 3 + 2] = make_float4(p[11], p[12], p[13], vf);
    tiles[item] = ntiles;
    depth[item] = tz32;
    dkey[item] = valid ? __float_as_uint(tz32) : 0xFFFFFFFFu;
    dval[item] = (uint32_t)item;
    return valid;
}

// One thread per (view, Gaussian) item; each CTA also writes how many of its 256
// consecutive items are visible (block_vis[view * gridDim.x + blockIdx.x]), the
// first step of the order-keeping compaction ahead of the depth sort, and the
// CTAs of view 0 the sum of their Gaussians' planar terms times reg_scale
// (reg_part[blockIdx.x]; the loss adds these partials in index order).
// Six CTAs of 256 threads per SM (at most 40 registers): 48 resident warps for a latency-bound
// per-thread chain (A/B on the 300k-Gaussian keyframe: iteration 0.5494 -> 0.5462 ms).
__global__ void __launch_bounds__(256, 6) k_preprocess(const float* __restrict__ P, int n, int cap,
                                                    const DevCamera* __restrict__ cams, DevConst kc, int tile,
                                                    float4* __restrict__ rec, uint32_t* __restrict__ tiles,
                                                    uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval,
                                                    float* __restrict__ depth, uint32_t* __restrict__ block_vis,
                                                    float reg_scale, float* __restrict__ reg_part) {
    __shared__ float wsum[8];
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int view = blockIdx.y;
    bool vis = false;
    float planar = 0.f;
    if (gid < n) vis = preprocess_one(P, n, cap, gid, view, cams, kc, tile, rec, tiles, dkey, dval, depth, planar);
    const int cnt = __syncthreads_count(vis);
    if (threadIdx.x == 0) block_vis[(size_t)view * gridDim.x + blockIdx.x] = (uint32_t)cnt;
    if (view == 0) {   // uniform over the CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) planar += __shfl_xor_sync(0xFFFFFFFFu, planar, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = planar;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < 8; ++w) t += wsum[w];
            reg_part[blockIdx.x] = t * reg_scale;
        }
    }
}

// Order-keeping compaction of the visible items, in item order, so that equal depths keep
// ascending ids through the stable sort. CTA B takes the items of projection CTAs 4B .. 4B + 3
// (linear index view * gx + x): it first adds the visible counts of the projection CTAs before
// them (a few thousand values at most, read straight from block_vis: no separate scan launch),
// then writes each one's visible keys and items in turn; the last CTA writes the total.
constexpr int kCompactSub = 4;
__global__ void __launch_bounds__(256) k_compact_visible(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin, int n, int gx,
                                                         int nblocks, const uint32_t* __restrict__ block_vis,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         uint32_t* __restrict__ total_out) {
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t s_off;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b0 = blockIdx.x * kCompactSub;
    {
        uint32_t pre = 0;
        for (int b = threadIdx.x; b < b0; b += 256) pre += block_vis[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
        if (lane == 0) wsum[w] = pre;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int k = 0; k < 8; ++k) t += wsum[k];
            s_off = t;
        }
        __syncthreads();
    }
    uint32_t off = s_off;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (int j = 0; j < kCompactSub && b0 + j < nblocks; ++j) {
        const int b = b0 + j, view = b / gx, gid = (b - view * gx) * 256 + threadIdx.x;
        const size_t item = (size_t)view * n + gid;
        const uint32_t key = gid < n ? kin[item] : 0xFFFFFFFFu;
        const bool vis = key != 0xFFFFFFFFu;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, vis);
        __syncthreads();   // the previous sub-block's counts have been read
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        uint32_t pre = 0, cnt = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            pre += k < w ? wsum[k] : 0u;
            cnt += wsum[k];
        }
        if (vis) {
            const uint32_t pos = off + pre + __popc(bal & lt);
            kout[pos] = key;
            vout[pos] = vin[item];
        }
        off += cnt;
    }
    if (total_out != nullptr && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = off;
}

// Six CTAs of 128 threads per SM (at most 85 registers): the kernel is latency-bound on its
// per-thread chain, and 24 resident warps instead of 20 beat the few spilled registers
// (A/B on the 300k-Gaussian keyframe: iteration 0.550 -> 0.545 ms; eight CTAs 0.548 ms).
__global__ void __launch_bounds__(128, 6) k_preprocess_backward(
    const float* __restrict__ P, int n, int cap, int n_views, const DevCamera* __restrict__ cams, DevConst kc,
    const float* __restrict__ grad2d, const uint32_t* __restrict__ tiles, float* __restrict__ G,
    float* __restrict__ dens_sum, float* __restrict__ dens_cnt, int add_reg, float reg_scale) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n) return;
    float p[kParamRows];
    load_params(P, cap, gid, p);
    float dmu[3] = {0.f, 0.f, 0.f};
    float dS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // symmetric (G + G^T) of dL/dSigma
    float dop = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
    float gsum = 0.f, gcnt = 0.f;
    Shape g;
    shape_of(p, g);
    Proj o;
    for (int view = 0; view < n_views; ++view) {
        size_t item = (size_t)view * n + gid;
        if (tiles[item] == 0) continue;
        const DevCamera& cam = cams[view];
        const float4 g0 = *reinterpret_cast<const float4*>(grad2d + item * kGrad2dStride);
        const float4 g1 = *reinterpret_cast<const float4*>(grad2d + item * kGrad2dStride + 4);
        const float g8 = grad2d[item * kGrad2dStride + 8];
        // the compositing adjoint leaves out the factor ln 2 of the first five values; with the
        // exp2 scaling of the conic (a' = -a log2(e) / 2, b' = -b log2(e)) it cancels there
        float gu = g0.x * kLn2, gv = g0.y * kLn2;
        float ga = -0.5f * g0.z, gb = -g0.w, gc = -0.5f * g1.x;   // to the unscaled conic
        dop += g1.y;
        dr += g1.z;
        dg += g1.w;
        db += g8;
        {   // densification statistic: position-gradient norm in NDC (du/dx_ndc = W/2)
            const float nu = gu * (0.5f * (float)cam.width), nv = gv * (0.5f * (float)cam.height);
            gsum += sqrtf(nu * nu + nv * nv);
        }
        gcnt += 1.f;
        project_one(p, g, cam, kc.dilation, o);
        // conic (a, b, c) = inverse of [[A, B], [B, C]]
        float id2 = 1.0f / (o.det * o.det);
        float A = o.A, B = o.B, C = o.C;
        float gA = id2 * (-C * C * ga + B * C * gb - B * B * gc);
        float gB = id2 * (2.f * B * C * ga - (o.det + 2.f * B * B) * gb + 2.f * A * B * gc);
        float gC = id2 * (-B * B * ga + A * B * gb - A * A * gc);
        // dL/dSigma (symmetrised): 2 gA T0T0^T + gB (T0T1^T + T1T0^T) + 2 gC T1T1^T
        const float* T0 = o.T0;
        const float* T1 = o.T1;
        dS[0] += 2.f * gA * T0[0] * T0[0] + 2.f * gB * T0[0] * T1[0] + 2.f * gC * T1[0] * T1[0];
        dS[1] += 2.f * gA * T0[0] * T0[1] + gB * (T0[0] * T1[1] + T1[0] * T0[1]) + 2.f * gC * T1[0] * T1[1];
        dS[2] += 2.f * gA * T0[0] * T0[2] + gB * (T0[0] * T1[2] + T1[0] * T0[2]) + 2.f * gC * T1[0] * T1[2];
        dS[3] += 2.f * gA * T0[1] * T0[1] + 2.f * gB * T0[1] * T1[1] + 2.f * gC * T1[1] * T1[1];
        dS[4] += 2.f * gA * T0[1] * T0[2] + gB * (T0[1] * T1[2] + T1[1] * T0[2]) + 2.f * gC * T1[1] * T1[2];
        dS[5] += 2.f * gA * T0[2] * T0[2] + 2.f * gB * T0[2] * T1[2] + 2.f * gC * T1[2] * T1[2];
        // dL/dT0 = 2 gA Sigma T0 + gB Sigma T1 ; dL/dT1 = gB Sigma T0 + 2 gC Sigma T1
        float ST0[3], ST1[3];
        ST0[0] = g.S[0] * T0[0] + g.S[1] * T0[1] + g.S[2] * T0[2];
        ST0[1] = g.S[1] * T0[0] + g.S[3] * T0[1] + g.S[4] * T0[2];
        ST0[2] = g.S[2] * T0[0] + g.S[4] * T0[1] + g.S[5] * T0[2];
        ST1[0] = g.S[0] * T1[0] + g.S[1] * T1[1] + g.S[2] * T1[2];
        ST1[1] = g.S[1] * T1[0] + g.S[3] * T1[1] + g.S[4] * T1[2];
        ST1[2] = g.S[2] * T1[0] + g.S[4] * T1[1] + g.S[5] * T1[2];
        float dT0[3], dT1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dT0[k] = 2.f * gA * ST0[k] + gB * ST1[k];
            dT1[k] = gB * ST0[k] + 2.f * gC * ST1[k];
        }
        // T = J W with rows T0 = J00 W0 + J02 W2, T1 = J11 W1 + J12 W2
        float dJ00 = dT0[0] * cam.R[0] + dT0[1] * cam.R[1] + dT0[2] * cam.R[2];
        float dJ02 = dT0[0] * cam.R[6] + dT0[1] * cam.R[7] + dT0[2] * cam.R[8];
        float dJ11 = dT1[0] * cam.R[3] + dT1[1] * cam.R[4] + dT1[2] * cam.R[5];
        float dJ12 = dT1[0] * cam.R[6] + dT1[1] * cam.R[7] + dT1[2] * cam.R[8];
        float iz = 1.0f / o.tz, iz2 = iz * iz, iz3 = iz2 * iz;
        float dtx = 0.f, dty = 0.f, dtz = 0.f;
        dtz += -cam.fx * iz2 * dJ00 - cam.fy * iz2 * dJ11;
        if (fabsf(o.xr) <= cam.lim_x) {
            dtx += -cam.fx * iz2 * dJ02;
            dtz += 2.f * cam.fx * o.tx * iz3 * dJ02;
        } else {
            dtz += cam.fx * o.xh * iz2 * dJ02;
        }
        if (fabsf(o.yr) <= cam.lim_y) {
            dty += -cam.fy * iz2 * dJ12;
            dtz += 2.f * cam.fy * o.ty * iz3 * dJ12;
        } else {
            dtz += cam.fy * o.yh * iz2 * dJ12;
        }
        // screen mean u = fx tx/tz + cx, v = fy ty/tz + cy
        dtx += gu * cam.fx * iz;
        dty += gv * cam.fy * iz;
        dtz += -(gu * cam.fx * o.tx + gv * cam.fy * o.ty) * iz2;
        // t = W mu + t_w
        dmu[0] += cam.R[0] * dtx + cam.R[3] * dty + cam.R[6] * dtz;
        dmu[1] += cam.R[1] * dtx + cam.R[4] * dty + cam.R[7] * dtz;
        dmu[2] += cam.R[2] * dtx + cam.R[5] * dty + cam.R[8] * dtz;
    }
    // Sigma = M M^T with M = R S: dL/dM = dS M
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[i * 3 + k] = g.R[i * 3 + k] * g.s[k];
    const float Sf[9] = {dS[0], dS[1], dS[2], dS[1], dS[3], dS[4], dS[2], dS[4], dS[5]};
    float dM[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dM[i * 3 + k] = Sf[i * 3 + 0] * M[0 * 3 + k] + Sf[i * 3 + 1] * M[1 * 3 + k] + Sf[i * 3 + 2] * M[2 * 3 + k];
    float dls[3];
    float dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ds = dM[0 * 3 + k] * g.R[0 * 3 + k] + dM[1 * 3 + k] * g.R[1 * 3 + k] + dM[2 * 3 + k] * g.R[2 * 3 + k];
        dls[k] = ds * g.s[k];
#pragma unroll
        for (int i = 0; i < 3; ++i) dR[i * 3 + k] = dM[i * 3 + k] * g.s[k];
    }
    if (add_reg) {
        // Eq. 10 planar term: mean_i max(floor, min_k s_ik); gradient on the (first) smallest axis
        int km = 0;
        float sm = g.s[0];
        if (g.s[1] < sm) { sm = g.s[1]; km = 1; }
        if (g.s[2] < sm) { sm = g.s[2]; km = 2; }
        if (sm > kc.reg_floor) dls[km] += reg_scale * sm;
    }
    // rotation of the normalised quaternion (w, x, y, z)
    float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
    float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    float dx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                      2.f * x * dR[8]);
    float dy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                      2.f * y * dR[8]);
    float dz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                      x * dR[6] + y * dR[7]);
    // through the normalisation q / |q|
    float dot = w * dw + x * dx + y * dy + z * dz;
    float iq = 1.0f / g.qnorm;
    float oa = 1.0f / (1.0f + expf(-p[10]));
    size_t c = (size_t)cap;
    G[0 * c + gid] = dmu[0];
    G[1 * c + gid] = dmu[1];
    G[2 * c + gid] = dmu[2];
    G[3 * c + gid] = dls[0];
    G[4 * c + gid] = dls[1];
    G[5 * c + gid] = dls[2];
    G[6 * c + gid] = (dw - w * dot) * iq;
    G[7 * c + gid] = (dx - x * dot) * iq;
    G[8 * c + gid] = (dy - y * dot) * iq;
    G[9 * c + gid] = (dz - z * dot) * iq;
    G[10 * c + gid] = dop * oa * (1.f - oa);
    G[11 * c + gid] = dr;
    G[12 * c + gid] = dg;
    G[13 * c + gid] = db;
    if (dens_sum != nullptr && gcnt > 0.f) {
        dens_sum[gid] += gsum;
        dens_cnt[gid] += gcnt;
    }
}

}  // namespace

// Projection of every (view, Gaussian) item, then the visible items compacted in
// item order into dkey[0] / dval[0] (their number in dcount[8]).
cudaError_t launch_preprocess(gs_ctx* c, int n_views, const DevConst& k, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    dim3 grid((c->n + 255) / 256, n_views);
    const uint32_t nblocks = grid.x * grid.y;
    c->launches += 2;
    k_preprocess<<<grid, 256, 0, s>>>(c->params, c->n, c->cap, c->dcam, k, c->tile, c->rec, c->tiles_touched,
                                       c->dkey[1], c->dval[1], c->depth, c->vis_blocks,
                                       k.lambda_reg / (float)c->n, c->reg_part);
    k_compact_visible<<<(nblocks + kCompactSub - 1) / kCompactSub, 256, 0, s>>>(
        c->dkey[1], c->dval[1], c->n, (int)grid.x, (int)nblocks, c->vis_blocks, c->dkey[0], c->dval[0], c->dcount + 8);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(gs_ctx* c, const DevConst& k, bool add_reg, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    float reg_scale = k.lambda_reg / (float)c->n;
    ++c->launches;
    k_preprocess_backward<<<(c->n + 127) / 128, 128, 0, s>>>(c->params, c->n, c->cap, c->n_views, c->dcam, k,
                                                              c->grad2d, c->tiles_touched, c->grads, c->dens_sum,
                                                              c->dens_cnt, add_reg ? 1 : 0, reg_scale);
    return cudaGetLastError();
}

}  // namespace gs
