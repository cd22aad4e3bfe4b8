// Front-to-back alpha compositing (Eq. 3, Section 3.1) and its adjoint.
//
// A persistent grid walks the (view, tile) work list; each thread owns PPT
// pixels of one column of its tile, and each warp an 8 x (4 PPT) pixel block, so
// a Gaussian that misses a warp's block costs that warp one test. The tile's
// sorted pair list is walked in batches of records staged in shared memory
// (gathered by Gaussian id from the 48-byte raster records).
//
// Membership is pixel-exact (|px - u| <= r and |py - v| <= r), so the image is
// the same for every tile size: tiles only bound which Gaussians a pixel tests.
#include <algorithm>
#include <type_traits>

#include "gs_internal.cuh"

namespace gs {
namespace {

// records staged in shared memory per batch: 512 for CTAs of 128 or 256
// threads (fewer barriers per tile: on the 300k-Gaussian keyframe 2 % faster
// than 256 for 256 threads, 3 % for 128; 128 records were 7 % slower), 256 for
// CTAs of 64 threads (there 512 records limit the SM to 6 CTAs by shared memory
// and the 8-view window slows by 30 %)
constexpr int batch_for(int threads) { return threads >= 128 ? 512 : 256; }

// A Gaussian that at most this many lanes of a warp blended gets its 9
// gradient values added by each of those lanes (two float4 atomics and one
// scalar) instead of a 12-shuffle warp sum and one 9-lane atomic: fewer issue
// slots for the warp; past about half a warp the same-address atomics cost more
// (on the 300k-Gaussian keyframe, 16 x 2 layout: 7 % faster than a threshold of
// one lane, 24 about 1 % faster than 16 and 12; every lane, 2 % slower)
constexpr int kLaneAtomicMax = 24;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


// A raster record staged for one tile, relative to the local origin (ox, oy),
// the tile's corner rounded down to a multiple of 32 px:
//   s0 = {u, v, hx, hy}: local screen mean and the half-widths of the pixel
//        box a pixel must lie in to be blended;
//   s1 = {a', b', c', o}: exp2-scaled conic and opacity;
//   s2 = {R, G, B, thr}: colour and the exponent threshold of the alpha cutoff.
// The screen mean is stored split (integer part in f0.xy, fractions in f1.w,
// f2.w); the local mean (ui - ox) + uf is formed once per pair and tile, so
// pixel offsets carry the rounding of a small number only, and the same for
// tiles of 8, 16 or 32 px (which keeps the image bit-identical across tile
// sizes).
//
// Blending needs |dx| <= r, |dy| <= r (the membership box) and
// o 2^p2 >= alpha_min, i.e. p2 >= thr = log2(alpha_min / o) with
// p2 = a' dx^2 + b' dx dy + c' dy^2 (negative definite). The set p2 >= thr is
// an ellipse whose axis-aligned half-widths are sqrt(-thr (B^-1)_xx),
// sqrt(-thr (B^-1)_yy) with B = -[[a', b'/2], [b'/2, c']]; hx, hy are those
// widths enlarged by 0.1 % + 0.01 px (far above float32 rounding) and capped
// at r, so a pixel outside (hx, hy) cannot blend and skipping it leaves the
// result unchanged. A Gaussian with o < alpha_min gets hx = hy = -1.
__device__ __forceinline__ void stage_record(const float4* __restrict__ rec, uint32_t item, float ox, float oy,
                                             float alpha_min, float4& s0, float4& s1, float4& s2) {
    const float4 a = rec[(size_t)item * 3 + 0];
    const float4 q = rec[(size_t)item * 3 + 1];
    const float4 c = rec[(size_t)item * 3 + 2];
    const float r = a.z, o = a.w;
    const float thr = log2f(alpha_min) - log2f(o);
    float hx = -1.f, hy = -1.f;
    if (thr <= 0.f) {
        const float det = q.x * q.z - 0.25f * q.y * q.y;
        if (det > 0.f) {
            const float kap = -thr / det;
            hx = fminf(fmaf(sqrtf(-kap * q.z), 1.001f, 0.01f), r);
            hy = fminf(fmaf(sqrtf(-kap * q.x), 1.001f, 0.01f), r);
        } else {
            hx = hy = r;
        }
    }
    s0 = make_float4((a.x - ox) + q.w, (a.y - oy) + c.w, hx, hy);
    s1 = make_float4(q.x, q.y, q.z, o);
    s2 = make_float4(c.x, c.y, c.z, thr);
}

// The same ellipse's extent across its long axis: with Q = -(a' dx^2 + b' dx dy + c' dy^2)
// = d^T M d, the set Q <= -thr has half-width sqrt(-thr / lambda_max(M)) along the unit
// eigenvector n of lambda_max(M) (the ellipse's short axis), enlarged by the same margin as the
// box. A pixel block whose projection on n lies farther from the mean cannot blend; for an
// elongated, rotated ellipse this strip cuts much of its axis-aligned box.
__device__ __forceinline__ void short_axis_strip(const float4 s1, float thr, float& nx, float& ny, float& wn) {
    nx = 1.f;
    ny = 0.f;
    wn = 3.0e38f;
    const float A = -s1.x, B2 = -0.5f * s1.y, C = -s1.z;   // M = [[A, B2], [B2, C]]
    if (!(thr <= 0.f)) return;
    const float half = 0.5f * (A - C);
    const float lam = 0.5f * (A + C) + sqrtf(half * half + B2 * B2);
    if (!(lam > 0.f)) return;
    // eigenvector of lam: the better conditioned of (B2, lam - A) and (lam - C, B2)
    float ex = B2, ey = lam - A;
    const float fx = lam - C, fy = B2;
    if (fx * fx + fy * fy > ex * ex + ey * ey) {
        ex = fx;
        ey = fy;
    }
    const float nn = ex * ex + ey * ey;
    if (!(nn > 0.f)) return;
    const float inv = rsqrtf(nn);
    nx = ex * inv;
    ny = ey * inv;
    wn = fmaf(sqrtf(-thr / lam), 1.001f, 0.01f);
}

// Thread layout of a TILE x TILE tile: each thread owns PPT pixels of one
// column, 4 rows apart; warp w owns an 8 x (4 PPT) block.
template <int TILE, int PPT>
struct Layout {
    static constexpr int kThreads = TILE * TILE / PPT;
    static constexpr int kBlocksX = TILE / 8;
    // resident CTAs per SM the fused kernel is compiled for (its register cap): 16 x 1 (8 warps a
    // CTA) capped at 64 registers for 4 CTAs instead of 3 (8-view 640x480 window: fused kernel
    // 0.748 -> 0.645 ms; 5 CTAs 0.652, 6 CTAs 0.716). 0 leaves the bound unset, so the others
    // keep the compiler's own register count (an explicit bound of 1 let it take more: 16 x 2
    // rose from 80 to 96 registers, 5 CTAs per SM instead of 6, 5 % slower)
    static constexpr int kMinBlocks = (TILE == 16 && PPT == 1) ? 4 : 0;
    // the adjoint reuses the forward's staged batch and visit lists when the tile's whole list
    // fits one batch, and then starts without CTA barriers (each warp cuts its own list at its
    // own end): 16 x 1 window 0.645 -> 0.634 ms, 8 x 1 0.653 -> 0.636 ms; not for 16 x 2, where
    // the warps' imbalance moves to the work queue's barrier (300k-Gaussian keyframe: 0.362 ->
    // 0.383 ms)
    static constexpr bool kReuseStaged = !(TILE == 16 && PPT == 2);
    __device__ static void pixel(int tid, int& lx, int& ly0) {
        const int w = tid >> 5, l = tid & 31;
        lx = (w % kBlocksX) * 8 + (l & 7);
        ly0 = (w / kBlocksX) * (4 * PPT) + (l >> 3);
    }
};

// Base-2 exponent a' dx^2 + b' dx dy + c' dy^2 of a Gaussian at a pixel, as a
// polynomial in dy: (c' dy + b' dx) dy + a' dx^2, with the column terms
// b' dx and a' dx^2 formed once per (thread, Gaussian) and shared by the
// thread's pixels; two fused multiply-adds per pixel. Written with explicit
// rounding so that every kernel takes bit-identical decisions.
__device__ __forceinline__ float power2_dy(float qz, float qydx, float qxdx2, float dy) {
    return __fmaf_rn(__fmaf_rn(qz, dy, qydx), dy, qxdx2);
}

// Warp sum of 9 values by recursive halving: at each step a lane keeps half of
// its values and trades the other half with its partner, so 9 values cost 11
// exchanges instead of 45. Afterwards even lane L holds the full sum of value
// *idx (or idx = -1 if its slot is padding); each value sits in exactly one
// even lane.
__device__ __forceinline__ float warp_sum9(const float (&v)[9], int lane, int& idx) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float w[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float a = v[i], b = (i + 5 < 9) ? v[i + 5] : 0.f;
        w[i] = (b4 ? b : a) + __shfl_xor_sync(0xFFFFFFFFu, b4 ? a : b, 16);
    }
    float x[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float a = w[i], b = (i + 3 < 5) ? w[i + 3] : 0.f;
        x[i] = (b3 ? b : a) + __shfl_xor_sync(0xFFFFFFFFu, b3 ? a : b, 8);
    }
    float y[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float a = x[i], b = (i + 2 < 3) ? x[i + 2] : 0.f;
        y[i] = (b2 ? b : a) + __shfl_xor_sync(0xFFFFFFFFu, b2 ? a : b, 4);
    }
    float z = (b1 ? y[1] : y[0]) + __shfl_xor_sync(0xFFFFFFFFu, b1 ? y[0] : y[1], 2);
    z += __shfl_xor_sync(0xFFFFFFFFu, z, 1);
    const int s3 = b2 ? 2 : 0, s4 = b1 ? 1 : 0;
    const int local = (b3 ? 3 : 0) + s3 + s4;
    const int id = (b4 ? 5 : 0) + local;
    idx = ((lane & 1) == 0 && s3 + s4 < 3 && local < 5 && id < 9) ? id : -1;
    return z;
}

// Shared-memory staging of one batch of B raster records for a CTA of NW
// warps, shared by the forward and backward passes.
template <int B, int NW>
struct Stage {
    // index of an entry of a staged batch
    typedef typename std::conditional<B <= 256, uint8_t, uint16_t>::type Idx;
    float4 s0[B], s1[B], s2[B];
    uint32_t sid[B];
    uint32_t mask[B];   // bit w: the record's pixel box meets warp w's pixel block
    Idx list[NW][B];   // per warp: the batch entries it must visit, in order
};

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Compacts the entries k < cnt of the staged batch whose mask has this warp's
// bit (and, when `limit` is given, lie before it) into the warp's list, in
// ascending order; returns their number. Called by all 32 lanes of the warp.
template <int B, int NW>
__device__ __forceinline__ int build_warp_list(Stage<B, NW>& st, int cnt, uint32_t base, uint32_t limit) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t wbit = 1u << w, lt = lanemask_lt();
    int nk = 0;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int k = c0 + lane;
        const bool hit = k < cnt && (st.mask[k] & wbit) && base + (uint32_t)k < limit;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hit);
        if (hit) st.list[w][nk + __popc(bal & lt)] = (typename Stage<B, NW>::Idx)k;
        nk += __popc(bal);
    }
    __syncwarp();
    return nk;
}
template <int B, int NW>
__device__ __forceinline__ Stage<B, NW>& stage() {
    __shared__ Stage<B, NW> st;
    return st;
}

// Geometry of one work item (a tile of one view) as seen by one thread.
template <int TILE, int PPT>
struct TileGeom {
    int view, txi, tyi, px, py0;
    float ox, oy, fx;
    uint2 rg;
    __device__ TileGeom(int bin, const uint2* __restrict__ ranges, int tiles_x, int tiles_per_view) {
        view = bin / tiles_per_view;
        const int t = bin - view * tiles_per_view;
        tyi = t / tiles_x;
        txi = t - tyi * tiles_x;
        int lx, ly0;
        Layout<TILE, PPT>::pixel(threadIdx.x, lx, ly0);
        px = txi * TILE + lx;
        py0 = tyi * TILE + ly0;
        // pixel offsets are taken from a 32-px-aligned local origin (see load_record)
        ox = (float)((txi * TILE) & ~31);
        oy = (float)((tyi * TILE) & ~31);
        fx = (float)px - ox;
        rg = ranges[bin];
    }
    __device__ int py(int p) const { return py0 + 4 * p; }
};

// Warps of the CTA whose 8 x (4 PPT) pixel block meets the box u +- hx, v +- hy and the
// short-axis strip |n . (x - u)| <= wn.
template <int TILE, int PPT>
__device__ __forceinline__ uint32_t warp_mask(const TileGeom<TILE, PPT>& g, const float4 s0, const float4 s1,
                                              float thr) {
    float nx, ny, wn;
    short_axis_strip(s1, thr, nx, ny, wn);
    // half-extents of a warp's pixel block projected on n, plus the rounding slack of the box test
    const float hb = 3.5f * fabsf(nx) + 0.5f * (float)(4 * PPT - 1) * fabsf(ny) + wn + 0.01f;
    constexpr int NW = Layout<TILE, PPT>::kThreads / 32;
    constexpr int BX = Layout<TILE, PPT>::kBlocksX;
    const float tox = (float)(g.txi * TILE) - g.ox, toy = (float)(g.tyi * TILE) - g.oy;
    // widened by 0.01 px so that rounding cannot drop a pixel the per-pixel test would keep
    const float x0 = s0.x - s0.z - 0.01f, x1 = s0.x + s0.z + 0.01f, y0 = s0.y - s0.w - 0.01f,
                y1 = s0.y + s0.w + 0.01f;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const float bx = tox + 8.f * (float)(w % BX), by = toy + (float)(4 * PPT) * (float)(w / BX);
        const float sc = nx * (bx + 3.5f - s0.x) + ny * (by + 0.5f * (float)(4 * PPT - 1) - s0.y);
        const bool hit = x0 <= bx + 7.f && x1 >= bx && y0 <= by + (float)(4 * PPT - 1) && y1 >= by && fabsf(sc) <= hb;
        m |= hit ? (1u << w) : 0u;
    }
    return m;
}

// Forward compositing (Eq. 3) of a thread's PPT pixels over the tile's sorted
// list. Returns final T, the colour, and per pixel the number of list entries
// up to and including the last blended Gaussian; optionally the Eq. 8 argmax.
// The return value is the length of the warp's visit list when the tile's whole
// list was staged as one batch (it is left in shared memory for the adjoint),
// else -1; which of the two is the same for every warp of the CTA.
template <int TILE, int PPT, bool ARGMAX, bool DET>
__device__ __forceinline__ int fwd_core(const TileGeom<TILE, PPT>& g, const bool (&inside)[PPT],
                                         const uint32_t* __restrict__ pval, const uint32_t* __restrict__ emit_item,
                                         const float4* __restrict__ rec, const DevConst& kc, float (&T)[PPT], float (&cr)[PPT], float (&cg)[PPT],
                                         float (&cb)[PPT], uint32_t (&last)[PPT], uint32_t (&amax)[PPT]) {
    constexpr int NT = Layout<TILE, PPT>::kThreads;
    constexpr int kBatch = batch_for(NT);
    Stage<kBatch, NT / 32>& st = stage<kBatch, NT / 32>();
    float4* s0 = st.s0;
    float4* s1 = st.s1;
    float4* s2 = st.s2;
    uint32_t* sid = st.sid;
    // a pixel that is outside the image or has stopped gets a row offset so far away that it
    // fails every box test (and its exponent is -inf): no separate per-pixel flag to test
    constexpr float kGone = 3.0e38f;
    float fy[PPT], wmax[PPT];
    int nlive = 0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        fy[p] = inside[p] ? (float)g.py(p) - g.oy : kGone;
        nlive += inside[p] ? 1 : 0;
        T[p] = 1.f;
        cr[p] = cg[p] = cb[p] = 0.f;
        last[p] = 0;
        wmax[p] = -1.f;
        amax[p] = 0xFFFFFFFFu;
    }
    const uint2 rg = g.rg;
    int staged = -1;
    for (uint32_t bs = rg.x; bs < rg.y; bs += kBatch) {
        if (__syncthreads_count(nlive > 0) == 0) break;
        for (int i = threadIdx.x; i < kBatch; i += NT) {
            const uint32_t j = bs + i;
            if (j < rg.y) {
                const uint32_t pv = pval[j];   // the item, or its emission index (deterministic mode)
                const uint32_t item = DET ? emit_item[pv] : pv;
                stage_record(rec, item, g.ox, g.oy, kc.alpha_min, s0[i], s1[i], s2[i]);
                sid[i] = pv;
                st.mask[i] = warp_mask<TILE, PPT>(g, s0[i], s1[i], s2[i].w);
            }
        }
        __syncthreads();
        const int cnt = min((uint32_t)kBatch, rg.y - bs);
        const int nk = build_warp_list(st, cnt, 0u, 0xFFFFFFFFu);
        if (rg.y - rg.x <= (uint32_t)kBatch) staged = nk;
        const typename Stage<kBatch, NT / 32>::Idx* wl = st.list[threadIdx.x >> 5];
        int knext = nk > 0 ? (int)wl[0] : 0;   // the next entry's index is loaded one visit ahead
        // unrolled by two: the next entry's record loads and membership tests interleave with
        // this entry's blending (A/B on the 300k-Gaussian keyframe, 16 x 2 layout: fused kernel
        // 0.380 -> 0.362 ms; the other layouts and the window unchanged; by four no better)
#pragma unroll 2
        for (int i = 0; i < nk && nlive > 0; ++i) {
            const int k = knext;
            if (i + 1 < nk) knext = wl[i + 1];
            const float4 a = s0[k];
            const float dx = g.fx - a.x;
            if (fabsf(dx) > a.z) continue;
            const float4 q = s1[k];
            const float thr = s2[k].w;
            const float qydx = __fmul_rn(q.y, dx), qxdx2 = __fmul_rn(__fmul_rn(q.x, dx), dx);
            // exponent and membership of every pixel first, without branches, so the
            // pixels' dependent chains interleave (5 % on the 300k-Gaussian keyframe
            // together with the same split in the adjoint)
            float p2v[PPT];
            bool hit[PPT];
            bool any_hit = false;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const float dy = fy[p] - a.y;
                p2v[p] = power2_dy(q.z, qydx, qxdx2, dy);
                hit[p] = fabsf(dy) <= a.w && p2v[p] >= thr;
                any_hit |= hit[p];
            }
            if (!any_hit) continue;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                if (!hit[p]) continue;
                const float alpha = fminf(kc.alpha_max, __fmul_rn(q.w, ex2_approx(p2v[p])));
                const float Tn = __fmul_rn(T[p], 1.f - alpha);
                if (Tn < kc.T_min) {
                    fy[p] = kGone;
                    --nlive;
                    continue;
                }
                const float wgt = alpha * T[p];
                const float4 c = s2[k];
                cr[p] = fmaf(c.x, wgt, cr[p]);
                cg[p] = fmaf(c.y, wgt, cg[p]);
                cb[p] = fmaf(c.z, wgt, cb[p]);
                T[p] = Tn;
                last[p] = bs + k - rg.x + 1;
                if (ARGMAX && wgt > wmax[p]) {
                    wmax[p] = wgt;
                    amax[p] = DET ? emit_item[sid[k]] : sid[k];
                }
            }
        }
    }
    return staged;
}

// Adjoint of the compositing for a thread's PPT pixels: walks the tile's list
// back to front from the block's largest last-blended entry, recovering
// T_i = T_{i+1} / (1 - alpha_i) from the final T, and accumulates the
// gradients w.r.t. each Gaussian's screen quantities (the first five, u, v and
// the exp2-scaled conic a', b', c', without the factor ln 2 of d 2^p / dp) (when at most
// kLaneAtomicMax lanes blended it, each adds its own 9 values with two float4
// atomics and one scalar; else a warp sum, then one 9-lane atomic). Each
// warp visits only the batch entries its compacted list holds, which stop at
// the warp's largest last-blended entry. With staged >= 0 (the forward left the
// tile's whole list staged, and this warp's visit list of that length) each
// warp cuts its own list at its own end and walks it without a CTA barrier.
template <int TILE, int PPT, bool DET>
__device__ __forceinline__ void bwd_core(const TileGeom<TILE, PPT>& g, const uint32_t* __restrict__ pval,
                                         const uint32_t* __restrict__ emit_item, const float4* __restrict__ rec,
                                         const DevConst& kc, float (&T)[PPT], const uint32_t (&cnt_last)[PPT],
                                         const float (&gr)[PPT], const float (&gg)[PPT], const float (&gb)[PPT],
                                         float* __restrict__ grad2d, float* __restrict__ pairgrad, int staged,
                                         bool fwd_masks) {
    constexpr int NT = Layout<TILE, PPT>::kThreads;
    constexpr int kBatch = batch_for(NT);
    Stage<kBatch, NT / 32>& st = stage<kBatch, NT / 32>();
    float4* s0 = st.s0;
    float4* s1 = st.s1;
    float4* s2 = st.s2;
    uint32_t* sid = st.sid;
    __shared__ uint32_t smax;
    const int lane = threadIdx.x & 31;
    const uint2 rg = g.rg;
    float fy[PPT], ga[PPT];   // ga: upstream gradient . normalised colour behind the current Gaussian
    uint32_t my_end[PPT];
    uint32_t thread_end = rg.x;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        fy[p] = (float)g.py(p) - g.oy;
        ga[p] = 0.f;
        my_end[p] = rg.x + cnt_last[p];
        thread_end = max(thread_end, my_end[p]);
    }
    const uint32_t wm = __reduce_max_sync(0xFFFFFFFFu, thread_end);
    uint32_t end = wm;
    if (staged < 0) {   // the CTA's largest end decides which batches are staged again
        __syncthreads();
        if (threadIdx.x == 0) smax = rg.x;
        __syncthreads();
        if (lane == 0) atomicMax(&smax, wm);
        __syncthreads();
        end = smax;
    }
    const uint32_t warp_end = wm;
    for (uint32_t be = end; be > rg.x;) {
        const uint32_t bs = be - rg.x > (uint32_t)kBatch ? be - kBatch : rg.x;
        const typename Stage<kBatch, NT / 32>::Idx* wl = st.list[threadIdx.x >> 5];
        int nk;
        if (staged >= 0) {
            // the forward's visit list (ascending) is still staged: cut it before the warp's end
            int lo = 0, hi = staged;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (bs + (uint32_t)wl[mid] < warp_end) lo = mid + 1;
                else hi = mid;
            }
            nk = lo;
        } else {
            // the forward's warp masks of a one-batch tile are still staged (nothing writes them
            // in between): only the records are staged again
            const bool keep_masks = fwd_masks && rg.y - rg.x <= (uint32_t)kBatch;
            __syncthreads();
            for (int i = threadIdx.x; i < kBatch; i += NT) {
                const uint32_t j = bs + i;
                if (j < be) {
                    const uint32_t pv = pval[j];   // the item, or its emission index (deterministic mode)
                    const uint32_t item = DET ? emit_item[pv] : pv;
                    stage_record(rec, item, g.ox, g.oy, kc.alpha_min, s0[i], s1[i], s2[i]);
                    sid[i] = pv;
                    if (!keep_masks) st.mask[i] = warp_mask<TILE, PPT>(g, s0[i], s1[i], s2[i].w);
                }
            }
            __syncthreads();
            nk = build_warp_list(st, (int)(be - bs), bs, warp_end);
        }
        int knext = nk > 0 ? (int)wl[nk - 1] : 0;   // as in the forward: one visit ahead
        for (int i = nk - 1; i >= 0; --i) {
            const int k = knext;
            if (i > 0) knext = wl[i - 1];
            const uint32_t pos = bs + k;
            const float4 a = s0[k];
            const float dx = g.fx - a.x;
            const bool col = fabsf(dx) <= a.z && pos < thread_end;
            float acc[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) acc[i] = 0.f;
            bool any = false;
            if (col) {
                const float4 q = s1[k];
                const float4 c = s2[k];
                const float qydx = __fmul_rn(q.y, dx), qxdx2 = __fmul_rn(__fmul_rn(q.x, dx), dx);
                float p2v[PPT];
                bool hit[PPT];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {   // as in the forward: all pixels' tests first
                    const float dy = fy[p] - a.y;
                    p2v[p] = power2_dy(q.z, qydx, qxdx2, dy);
                    hit[p] = pos < my_end[p] && fabsf(dy) <= a.w && p2v[p] >= c.w;
                }
                float Gv[PPT];   // all pixels' ex2 back to back (the MUFU pipe has room)
#pragma unroll
                for (int p = 0; p < PPT; ++p) Gv[p] = ex2_approx(p2v[p]);
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    if (!hit[p]) continue;
                    const float dy = fy[p] - a.y;
                    const float G = Gv[p];
                    const float oG = __fmul_rn(q.w, G);
                    const float alpha = fminf(kc.alpha_max, oG);
                    any = true;
                    const float oma = 1.f - alpha;       // >= 1 - alpha_max = 0.01
                    T[p] = __fdividef(T[p], oma);        // transmittance in front of this Gaussian (2 ulp)
                    const float wgt = alpha * T[p];
                    acc[6] = fmaf(gr[p], wgt, acc[6]);
                    acc[7] = fmaf(gg[p], wgt, acc[7]);
                    acc[8] = fmaf(gb[p], wgt, acc[8]);
                    // dL/dalpha = T (g . c - g . a), with a the normalised colour behind this
                    // Gaussian, a <- a + alpha (c - a); g is fixed per pixel, so only g . a is kept
                    const float d = fmaf(gr[p], c.x, fmaf(gg[p], c.y, gb[p] * c.z)) - ga[p];
                    const float dalpha = T[p] * d;
                    ga[p] = fmaf(alpha, d, ga[p]);
                    // through alpha = o 2^p2, zero where the 0.99 clamp holds; the factor ln 2
                    // of d(2^p2)/dp2 is left to the readers of the screen gradients
                    const bool open = oG <= kc.alpha_max;
                    const float g2 = open ? dalpha * oG : 0.f;
                    acc[0] -= g2 * (2.f * q.x * dx + q.y * dy);
                    acc[1] -= g2 * (q.y * dx + 2.f * q.z * dy);
                    acc[2] = fmaf(g2 * dx, dx, acc[2]);
                    acc[3] = fmaf(g2 * dx, dy, acc[3]);
                    acc[4] = fmaf(g2 * dy, dy, acc[4]);
                    acc[5] = fmaf(dalpha, open ? G : 0.f, acc[5]);
                }
            }
            const uint32_t who = __ballot_sync(0xFFFFFFFFu, any);
            if (who == 0u) continue;
            if constexpr (DET) {
                // deterministic mode (one warp per tile): the warp's fixed-order sum is the
                // whole tile's contribution; it goes to the pair's own slot, no atomics
                int idx;
                const float v = warp_sum9(acc, lane, idx);
                if (idx >= 0) pairgrad[(size_t)sid[k] * kPairGradStride + idx] = v;
                continue;
            }
            if (__popc(who) <= kLaneAtomicMax) {
                // few lanes blended this Gaussian: each adds its own values (no warp sum)
                if (any) {
                    float* gp = grad2d + (size_t)sid[k] * kGrad2dStride;
                    atomicAdd(reinterpret_cast<float4*>(gp), make_float4(acc[0], acc[1], acc[2], acc[3]));
                    atomicAdd(reinterpret_cast<float4*>(gp + 4), make_float4(acc[4], acc[5], acc[6], acc[7]));
                    atomicAdd(gp + 8, acc[8]);
                }
                continue;
            }
            int idx;
            const float v = warp_sum9(acc, lane, idx);
            if (idx >= 0) atomicAdd(grad2d + (size_t)sid[k] * kGrad2dStride + idx, v);
        }
        be = bs;
    }
}

// Persistent compositing kernels: a grid sized to the GPU's resident capacity
// walks the (view, tile) work list through an atomic counter, so the load
// stays balanced across tiles of very different cost and across the views of
// a window. `order` (optional) lists the bins in the order to take them.
__device__ __forceinline__ bool next_work(uint32_t* __restrict__ queue, uint32_t n_items,
                                          const uint32_t* __restrict__ order, int& bin) {
    __shared__ uint32_t s_work;
    __syncthreads();
    if (threadIdx.x == 0) s_work = atomicAdd(queue, 1u);
    __syncthreads();
    const uint32_t w = s_work;
    if (w >= n_items) return false;
    bin = order ? (int)order[w] : (int)w;
    return true;
}

template <int TILE, int PPT>
__device__ __forceinline__ void inside_mask(const TileGeom<TILE, PPT>& g, int width, int height, bool (&inside)[PPT]) {
#pragma unroll
    for (int p = 0; p < PPT; ++p) inside[p] = g.px < width && g.py(p) < height;
}

template <int TILE, int PPT, bool ARGMAX, bool DET>
__global__ void __launch_bounds__(Layout<TILE, PPT>::kThreads)
    k_raster_fwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ pval, const float4* __restrict__ rec,
                 int width, int height, int tiles_x, int tiles_per_view, int n, DevConst kc,
                 float* __restrict__ out_rgb, float* __restrict__ out_T, uint32_t* __restrict__ out_last,
                 int32_t* __restrict__ out_argmax, uint32_t* __restrict__ queue, uint32_t n_items,
                 const uint32_t* __restrict__ order, const uint32_t* __restrict__ emit_item) {
    int bin;
    const size_t HW = (size_t)width * height;
    while (next_work(queue, n_items, order, bin)) {
        const TileGeom<TILE, PPT> g(bin, ranges, tiles_x, tiles_per_view);
        bool inside[PPT];
        inside_mask(g, width, height, inside);
        float T[PPT], cr[PPT], cg[PPT], cb[PPT];
        uint32_t last[PPT], amax[PPT];
        fwd_core<TILE, PPT, ARGMAX, DET>(g, inside, pval, emit_item, rec, kc, T, cr, cg, cb, last, amax);
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if (!inside[p]) continue;
            const size_t pix = (size_t)g.py(p) * width + g.px;
            out_rgb[(size_t)g.view * 3 * HW + pix] = cr[p];
            out_rgb[(size_t)g.view * 3 * HW + HW + pix] = cg[p];
            out_rgb[(size_t)g.view * 3 * HW + 2 * HW + pix] = cb[p];
            out_T[g.view * HW + pix] = T[p];
            out_last[g.view * HW + pix] = last[p];
            if (ARGMAX)
                out_argmax[g.view * HW + pix] =
                    amax[p] == 0xFFFFFFFFu ? -1 : (int32_t)(amax[p] - (uint32_t)g.view * n);
        }
    }
}

template <int TILE, int PPT, bool DET>
__global__ void __launch_bounds__(Layout<TILE, PPT>::kThreads)
    k_raster_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ pval, const float4* __restrict__ rec,
                 int width, int height, int tiles_x, int tiles_per_view, DevConst kc,
                 const float* __restrict__ T_final, const uint32_t* __restrict__ n_last,
                 const float* __restrict__ dLdC, float* __restrict__ grad2d, uint32_t* __restrict__ queue,
                 uint32_t n_items, const uint32_t* __restrict__ order, const uint32_t* __restrict__ emit_item,
                 float* __restrict__ pairgrad) {
    int bin;
    const size_t HW = (size_t)width * height;
    while (next_work(queue, n_items, order, bin)) {
        const TileGeom<TILE, PPT> g(bin, ranges, tiles_x, tiles_per_view);
        float T[PPT], gr[PPT], gg[PPT], gb[PPT];
        uint32_t cnt[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            T[p] = 1.f;
            gr[p] = gg[p] = gb[p] = 0.f;
            cnt[p] = 0;
            if (g.px < width && g.py(p) < height) {
                const size_t pix = (size_t)g.py(p) * width + g.px;
                T[p] = T_final[g.view * HW + pix];
                cnt[p] = n_last[g.view * HW + pix];
                gr[p] = dLdC[(size_t)g.view * 3 * HW + pix];
                gg[p] = dLdC[(size_t)g.view * 3 * HW + HW + pix];
                gb[p] = dLdC[(size_t)g.view * 3 * HW + 2 * HW + pix];
            }
        }
        bwd_core<TILE, PPT, DET>(g, pval, emit_item, rec, kc, T, cnt, gr, gg, gb, grad2d, pairgrad, -1, false);
    }
}

// One mapping iteration's compositing for every (view, tile): forward (Eq. 3),
// the L1 term of Eq. 10 and dL/dC = lambda sign(C - I) / 3HW for the tile's
// pixels, then the adjoint, with final T, last index and dL/dC kept in
// registers. Writes the image and one photometric partial sum per CTA.
template <int TILE, int PPT, bool DET>
__global__ void __launch_bounds__(Layout<TILE, PPT>::kThreads, Layout<TILE, PPT>::kMinBlocks)
    k_raster_fused(const uint2* __restrict__ ranges, const uint32_t* __restrict__ pval,
                   const float4* __restrict__ rec, int width, int height, int tiles_x, int tiles_per_view,
                   DevConst kc, const float* __restrict__ target, const float* const* __restrict__ target_slot,
                   float scale, float* __restrict__ out_rgb, float* __restrict__ grad2d, float* __restrict__ partials,
                   uint32_t* __restrict__ queue, uint32_t n_items, const uint32_t* __restrict__ order,
                   const uint32_t* __restrict__ emit_item, float* __restrict__ pairgrad,
                   float* __restrict__ tile_part) {
    if (target_slot != nullptr) target = *target_slot;   // a replayed graph's per-call target
    int bin;
    const size_t HW = (size_t)width * height;
    float loss = 0.f;
    while (next_work(queue, n_items, order, bin)) {
        const TileGeom<TILE, PPT> g(bin, ranges, tiles_x, tiles_per_view);
        bool inside[PPT];
        inside_mask(g, width, height, inside);
        float T[PPT], cr[PPT], cg[PPT], cb[PPT], gr[PPT], gg[PPT], gb[PPT];
        uint32_t last[PPT], amax[PPT];
        const int staged =
            fwd_core<TILE, PPT, false, DET>(g, inside, pval, emit_item, rec, kc, T, cr, cg, cb, last, amax);
        float tl = 0.f;   // this thread's photometric sum over the tile
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            gr[p] = gg[p] = gb[p] = 0.f;
            if (!inside[p]) {
                last[p] = 0;
                continue;
            }
            const size_t pix = (size_t)g.py(p) * width + g.px;
            const size_t o = (size_t)g.view * 3 * HW + pix;
            out_rgb[o] = cr[p];
            out_rgb[o + HW] = cg[p];
            out_rgb[o + 2 * HW] = cb[p];
            const float r0 = cr[p] - target[o], r1 = cg[p] - target[o + HW], r2 = cb[p] - target[o + 2 * HW];
            tl += (fabsf(r0) + fabsf(r1)) + fabsf(r2);
            gr[p] = scale * (float)((r0 > 0.f) - (r0 < 0.f));
            gg[p] = scale * (float)((r1 > 0.f) - (r1 < 0.f));
            gb[p] = scale * (float)((r2 > 0.f) - (r2 < 0.f));
        }
        loss += tl;
        if constexpr (DET) {
            // deterministic mode: each tile's sum on its own (fixed tree), whichever CTA took it
            __shared__ float tred[32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tl += __shfl_xor_sync(0xFFFFFFFFu, tl, o);
            if ((threadIdx.x & 31) == 0) tred[threadIdx.x >> 5] = tl;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.f;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += tred[w];
                tile_part[bin] = t * scale;
            }
            __syncthreads();
        }
        bwd_core<TILE, PPT, DET>(g, pval, emit_item, rec, kc, T, last, gr, gg, gb, grad2d, pairgrad,
                                 (DET || !Layout<TILE, PPT>::kReuseStaged) ? -1 : staged, true);
    }
    // per-CTA photometric partial (already scaled)
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partials[blockIdx.x] = t * scale;
    }
}

// Algorithmic work of the last render, by replaying the forward traversal per
// pixel: out[0] += list entries the forward pass reaches (up to and including
// the stopping one), out[1] += pairs blended, out[2] += list entries the
// backward pass reaches (up to the last blended one).
template <int TILE>
__global__ void __launch_bounds__(TILE* TILE) k_count_work(const uint2* __restrict__ ranges,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ pval,
                                                           const uint32_t* __restrict__ emit_item, int width, int height,
                                                           int tiles_x, int tiles_per_view, DevConst kc,
                                                           unsigned long long* __restrict__ out) {
    const int bin = blockIdx.x;
    const int view = bin / tiles_per_view;
    const int t = bin - view * tiles_per_view;
    const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int px = txi * TILE + lx, py = tyi * TILE + ly;
    if (px >= width || py >= height) return;
    const float ox = (float)((txi * TILE) & ~31), oy = (float)((tyi * TILE) & ~31);
    const float fx = (float)px - ox, fy = (float)py - oy;
    const uint2 rg = ranges[bin];
    float T = 1.f;
    unsigned long long tested = 0, blended = 0, walked = 0;
    for (uint32_t j = rg.x; j < rg.y; ++j) {
        const uint32_t item = emit_item != nullptr ? emit_item[pval[j]] : pval[j];
        float4 a, q, c;
        stage_record(rec, item, ox, oy, kc.alpha_min, a, q, c);
        ++tested;
        const float dx = fx - a.x, dy = fy - a.y;
        if (fabsf(dx) > a.z || fabsf(dy) > a.w) continue;
        const float p2 = power2_dy(q.z, __fmul_rn(q.y, dx), __fmul_rn(__fmul_rn(q.x, dx), dx), dy);
        if (p2 < c.w) continue;
        const float alpha = fminf(kc.alpha_max, __fmul_rn(q.w, ex2_approx(p2)));
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
        k_count_work<16><<<c->n_bins, 256, 0, s>>>(c->ranges, c->rec, c->pval[c->pair_buf], c->emit_item, c->width,
                                                   c->height, c->hcam[0].tiles_x, tpv, k, out);
    else
        k_count_work<8><<<c->n_bins, 64, 0, s>>>(c->ranges, c->rec, c->pval[c->pair_buf], c->emit_item, c->width,
                                                 c->height, c->hcam[0].tiles_x, tpv, k, out);
    return cudaGetLastError();
}

// resident CTAs of a kernel on the whole GPU (cached per kernel instantiation)
template <int KIND, int TILE, int PPT, typename K>
static int resident_grid(K kernel, int threads, int num_sms) {
    static int cached = 0;
    if (cached == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        cached = per_sm * num_sms;
    }
    return cached;
}

template <int TILE, int PPT, bool DET>
static void fwd_launch(gs_ctx* c, const DevConst& k, float* rgb, int32_t* argmax, cudaStream_t s, int tpv) {
    constexpr int NT = Layout<TILE, PPT>::kThreads;
    if (argmax) {
        const int grid =
            std::min(resident_grid<0 + 4 * DET, TILE, PPT>(k_raster_fwd<TILE, PPT, true, DET>, NT, c->num_sms), c->n_bins);
        k_raster_fwd<TILE, PPT, true, DET><<<grid, NT, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                          c->hcam[0].tiles_x, tpv, c->n, k, rgb, c->T_final,
                                                          c->n_last, argmax, c->dcount + 6, (uint32_t)c->n_bins,
                                                          c->work_order, c->emit_item);
    } else {
        const int grid =
            std::min(resident_grid<1 + 4 * DET, TILE, PPT>(k_raster_fwd<TILE, PPT, false, DET>, NT, c->num_sms),
                     c->n_bins);
        k_raster_fwd<TILE, PPT, false, DET><<<grid, NT, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width,
                                                           c->height, c->hcam[0].tiles_x, tpv, c->n, k, rgb,
                                                           c->T_final, c->n_last, nullptr, c->dcount + 6,
                                                           (uint32_t)c->n_bins, c->work_order, c->emit_item);
    }
}

template <int TILE, int PPT, bool DET>
static void bwd_launch(gs_ctx* c, const DevConst& k, const float* dLdC, cudaStream_t s, int tpv) {
    constexpr int NT = Layout<TILE, PPT>::kThreads;
    const int grid =
        std::min(resident_grid<2 + 4 * DET, TILE, PPT>(k_raster_bwd<TILE, PPT, DET>, NT, c->num_sms), c->n_bins);
    k_raster_bwd<TILE, PPT, DET><<<grid, NT, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                c->hcam[0].tiles_x, tpv, k, c->T_final, c->n_last, dLdC, c->grad2d,
                                                c->dcount + 7, (uint32_t)c->n_bins, c->work_order, c->emit_item,
                                                c->pairgrad);
}

template <int TILE, int PPT, bool DET>
static void fused_launch(gs_ctx* c, const DevConst& k, const float* target, const float* const* target_slot,
                         float* rgb, cudaStream_t s, int tpv, float* partials, int max_grid, int* grid_out) {
    constexpr int NT = Layout<TILE, PPT>::kThreads;
    const int grid = std::min(
        std::min(resident_grid<3 + 4 * DET, TILE, PPT>(k_raster_fused<TILE, PPT, DET>, NT, c->num_sms), c->n_bins),
        max_grid);
    const float scale = k.lambda_color / (float)(3 * (size_t)c->width * c->height);
    k_raster_fused<TILE, PPT, DET><<<grid, NT, 0, s>>>(c->ranges, c->pval[c->pair_buf], c->rec, c->width, c->height,
                                                  c->hcam[0].tiles_x, tpv, k, target, target_slot, scale, rgb,
                                                  c->grad2d, partials,
                                                  c->dcount + 6, (uint32_t)c->n_bins, c->work_order, c->emit_item,
                                                  c->pairgrad, c->tile_part);
    *grid_out = grid;
}

// The deterministic mode has one layout (8-px tiles, 2 pixels per thread: one
// warp per tile); the default mode any of the five.
#define GS_DISPATCH(FN, ...)                                         \
    do {                                                             \
        if (c->cfg.deterministic) {                                  \
            FN<8, 2, true>(__VA_ARGS__);                             \
        } else if (c->tile == 16) {                                  \
            if (c->ppt == 1) FN<16, 1, false>(__VA_ARGS__);          \
            else if (c->ppt == 2) FN<16, 2, false>(__VA_ARGS__);     \
            else FN<16, 4, false>(__VA_ARGS__);                      \
        } else {                                                     \
            if (c->ppt == 1) FN<8, 1, false>(__VA_ARGS__);           \
            else FN<8, 2, false>(__VA_ARGS__);                       \
        }                                                            \
    } while (0)

cudaError_t launch_raster_forward(gs_ctx* c, const DevConst& k, float* rgb, int32_t* argmax, cudaStream_t s) {
    const int tpv = c->hcam[0].tiles_x * c->hcam[0].tiles_y;
    if (c->n_bins == 0) return cudaSuccess;
    // work queue (a mapping iteration zeroes it on its side stream)
    cudaError_t e = c->side_zeroed ? cudaSuccess : cudaMemsetAsync(c->dcount + 6, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    ++c->launches;
    GS_DISPATCH(fwd_launch, c, k, rgb, argmax, s, tpv);
    return cudaGetLastError();
}

cudaError_t launch_raster_backward(gs_ctx* c, const DevConst& k, const float* dLdC, cudaStream_t s) {
    const int tpv = c->hcam[0].tiles_x * c->hcam[0].tiles_y;
    if (c->n_bins == 0) return cudaSuccess;
    // work queue (a mapping iteration zeroes it on its side stream)
    cudaError_t e = c->side_zeroed ? cudaSuccess : cudaMemsetAsync(c->dcount + 7, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    ++c->launches;
    GS_DISPATCH(bwd_launch, c, k, dLdC, s, tpv);
    return cudaGetLastError();
}

cudaError_t launch_raster_fused(gs_ctx* c, const DevConst& k, const float* target, const float* const* target_slot,
                                float* rgb, float* partials, int max_grid, int* grid_out, cudaStream_t s) {
    const int tpv = c->hcam[0].tiles_x * c->hcam[0].tiles_y;
    *grid_out = 0;
    if (c->n_bins == 0) return cudaSuccess;
    // work queue (a mapping iteration zeroes it on its side stream)
    cudaError_t e = c->side_zeroed ? cudaSuccess : cudaMemsetAsync(c->dcount + 6, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    ++c->launches;
    GS_DISPATCH(fused_launch, c, k, target, target_slot, rgb, s, tpv, partials, max_grid, grid_out);
    return cudaGetLastError();
}

}  // namespace gs
