// Internal declarations of the GB300 splatting library: context layout, device
// camera record, launch wrappers. Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gs.h"

namespace gs {

constexpr int kParamRows = 14;
constexpr int kGrad2dStride = 12;   // floats per (view, Gaussian) screen-gradient record
constexpr int kPairGradStride = 9;  // floats per pair slot of the deterministic mode
constexpr int kRecFloat4 = 3;       // float4 per (view, Gaussian) raster record
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// largest pair buffer (pair indices are 32-bit)
constexpr int64_t kMaxPairs = 0xFFFFFFF0ll;

// Camera as the kernels read it (one per view, in device memory).
struct DevCamera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float lim_x, lim_y;     // fov_clamp * half-FOV tangents
    int width, height;
    int tiles_x, tiles_y;   // tiles of this view
    int bin_base;           // first bin index of this view
    int pad;
};

// Method constants as the kernels read them.
struct DevConst {
    float near_z, dilation, lambda_floor, radius_sigma;
    float alpha_min, alpha_max, T_min;
    float lambda_color, lambda_reg, reg_floor;
};

#ifdef __CUDACC__
// Pixel box |px - u| <= r, |py - v| <= r clipped to the image, from the split
// screen mean (integer part ui, fraction uf in [0, 1)): ceil(u) = ui + (uf > 0),
// floor(u) = ui. Exact in float for |ui| < 2^23 and r < 2^22. Shared by the
// tile count here and the pair emission so that both see the same box.
__device__ __forceinline__ bool pixel_box(float ui, float uf, float vi, float vf, float r, int width, int height,
                                          int& x0, int& x1, int& y0, int& y1) {
    float fx0 = fmaxf(ui + (uf > 0.f ? 1.f : 0.f) - r, 0.f), fx1 = fminf(ui + r, (float)(width - 1));
    float fy0 = fmaxf(vi + (vf > 0.f ? 1.f : 0.f) - r, 0.f), fy1 = fminf(vi + r, (float)(height - 1));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return false;
    x0 = (int)fx0;
    x1 = (int)fx1;
    y0 = (int)fy0;
    y1 = (int)fy1;
    return true;
}
#endif

}  // namespace gs

struct gs_ctx {
    gs_config cfg;
    int device = 0;
    int n = 0;                  // Gaussians in the map
    int cap = 0;                // capacity (Gaussians)
    int adam_t = 0;             // Adam steps taken
    double* adam_pw = nullptr;  // device {beta1^t, beta2^t} after t steps
    std::string err;

    // map state, [14][cap] planar
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* dens_sum = nullptr;  // [cap] sum of screen-space gradient norms
    float* dens_cnt = nullptr;  // [cap] number of visible backward passes
    uint32_t* dom_cnt = nullptr;  // [cap] dominated pixels counted by gs_count_dominant (Eq. 9)

    // per-render state
    int n_views = 0;            // views of the last render (0 = none)
    int width = 0, height = 0;  // size of every view of the last render
    int tile = 16;              // tile size of the last render
    int ppt = 4;                // pixels per thread of the compositing kernels (1, 2 or 4; 8-px tiles: 1 or 2)
    int n_bins = 0;             // bins of the last render
    gs::DevCamera hcam[GS_MAX_VIEWS];
    gs::DevCamera* dcam = nullptr;          // [max_views]
    float4* rec = nullptr;                  // [max_views * cap * 3]
    uint32_t* tiles_touched = nullptr;      // [max_views * cap]
    float* depth = nullptr;                 // [max_views * cap] float32 view depth
    uint32_t* dkey[2] = {nullptr, nullptr}; // depth-sort keys   [max_views * cap]
    uint32_t* dval[2] = {nullptr, nullptr}; // depth-sort values [max_views * cap]
    uint32_t* offsets = nullptr;            // exclusive scan of tiles touched in depth order
    int64_t pair_cap = 0;
    uint32_t* pkey[2] = {nullptr, nullptr}; // bin of each pair
    uint32_t* pval[2] = {nullptr, nullptr}; // (view * cap + id) of each pair
    int pair_buf = 0;                       // which of the two buffers holds the sorted pairs
    uint32_t pairs_hint = 0;                // host-side pair count of the last render (grid sizing)
    uint2* ranges = nullptr;                // [max bins] (start, end) per bin
    // deterministic mode only: the pairs' sort values are emission indices e; emit_item[e] is
    // the pair's (view, Gaussian) item and pairgrad[9 e ..] its screen-gradient slot
    uint32_t* emit_item = nullptr;          // [pair capacity]
    float* pairgrad = nullptr;              // [pair capacity * 9]
    float* tile_part = nullptr;             // [max bins] photometric loss per (view, tile)
    uint32_t* work_order = nullptr;         // [max bins] bins by decreasing pair count (while a
                                            // replay is captured: the graph's own buffer)
    int max_bins = 0;
    float* T_final = nullptr;               // [max_views * H * W]
    uint32_t* n_last = nullptr;             // [max_views * H * W] entries up to the last blended
    float* dLdC = nullptr;                  // [max_views * 3 * H * W]
    float* grad2d = nullptr;                // [max_views * cap * 12]
    const float* rendered_rgb = nullptr;    // caller buffer of the last render
    bool loss_ready = false;
    bool backward_ready = false;

    // scratch
    uint32_t* hist = nullptr;               // radix / scan block counters
    const float** target_slot = nullptr;    // device: the target image of the current iteration
    float* ssim_maps = nullptr;             // [3][V][3][H][W] SSIM derivative maps (lambda_photo > 0)
    float* ssim_part = nullptr;             // [2 ssim_blocks] per-CTA photometric loss terms
    int sort_blocks = 0;
    uint32_t* dcount = nullptr;             // device scalars [16]: [0] pairs, [1] overflow, [2] Adam
                                            // ticket, [3] UINT32_MAX, [4] Adam steps, [5] totals,
                                            // [6], [7] work queues, [8] visible (view, Gaussian) items,
                                            // [10] a non-finite loss or gradient was seen (sticky until
                                            // a call reports it)
    uint32_t* vis_blocks = nullptr;         // visible items per preprocess CTA, then their offsets
    uint32_t visible_hint = 0;              // host copy of dcount[8] from the last synchronising render
    uint32_t* hcount = nullptr;             // pinned host mirror
    float* partials = nullptr;              // reduction partials
    double* psnr_part = nullptr;            // [psnr_scratch_doubles()] partial sums of gs_psnr
    float* reg_part = nullptr;              // [ceil(cap / 256)] planar-term partials of the last projection
    float* fpart = nullptr;                 // photometric partials of the fused kernel (one per CTA)
    int n_fpart = 0;
    int n_partials = 0;
    int num_sms = 0;
    int64_t launches = 0;                   // kernels launched by this context

    // iterate() graph cache
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_src = nullptr;        // kept alive: exec updates address its nodes
    int graph_views = 0, graph_w = 0, graph_h = 0, graph_n = 0, graph_tile = 0, graph_ppt = 0;
    uint32_t graph_timing = 0;
    int64_t graph_pair_cap = 0;
    float* graph_loss = nullptr;
    float* graph_rgb = nullptr;
    cudaStream_t cap_stream = nullptr;      // stream the iteration is captured on
    // second stream of a mapping iteration: the zeroing it needs later runs there from its start,
    // overlapping the projection and the sorts, and the loss total runs there beside the
    // projection adjoint and Adam (a fork and joins, which a captured graph keeps as branches)
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev[6] = {};            // fork, overflow flag + ranges zeroed, grad2d zeroed,
                                            // second fork, side work done, ranges ready
    bool side_zeroed = false;               // this iteration's zeroing was issued on `side`
    // a replayed iteration composites in the longest-first order the previous one computed (any
    // order of the same bins gives the same result) and computes the next order on `side`
    bool order_ahead = false;
    uint32_t* work_order_next = nullptr;    // [max bins]
    uint32_t* work_order_graph = nullptr;   // [max bins] the order a replay composites in: its own
                                            // buffer, so that a render of another shape between
                                            // replays (which writes work_order) cannot change it
    cudaEvent_t graph_done = nullptr;       // recorded after each replay
    bool graph_pending = false;             // a replay's flags have not been checked yet
    uint32_t* hflags = nullptr;             // pinned [16]: dcount[0..10] as the last replay left them
    cudaGraphNode_t cam_node = nullptr;     // kernel node that uploads the cameras
    int64_t graph_kernels = 0;              // kernels per replay
    bool capturing = false;
    struct CapPhase {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<CapPhase> cap_phases;       // placeholder events recorded during capture
    struct TimedNode {
        int phase;
        cudaGraphNode_t a, b;
    };
    std::vector<TimedNode> graph_tnodes;    // event-record nodes around each phase
    float* own_rgb = nullptr;               // internal image when the caller gives none
    size_t own_rgb_elems = 0;
    // gs_iterate_host: the caller's host targets go up, alternately into two device buffers, on
    // `copy`; call k's upload waits for the start of call k-1's iteration on the caller's stream
    // (h2d_start) and the end of call k-2's (h2d_free, the last reader of its buffer), and call k's
    // iteration waits for it (h2d_ready): host-side stream waits only, so with the host ahead of the
    // device an upload runs beside the previous iteration
    cudaStream_t copy = nullptr;
    cudaEvent_t h2d_start[2] = {}, h2d_ready[2] = {}, h2d_free[2] = {};
    float* tgt_stage[2] = {};
    size_t tgt_stage_elems = 0;
    int h2d_k = 0;                          // buffer of the next call
    // phase timing (gs_timing_enable / gs_timing_read)
    uint32_t timing = 0;                 // bit p: phase p is timed
    struct TimingRec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<TimingRec> trec;
    std::vector<cudaEvent_t> tpool;
    // autotuned (tile size, pixels per thread) per (width, height, views, N-bucket)
    struct Tuned {
        int w, h, views, nb, tile, ppt;
    };
    std::vector<Tuned> tuned;
    int force_tile = 0, force_ppt = 0;      // set while the autotuner times a candidate
    gs_mlp* init_mlp = nullptr;             // learned initialiser of gs_insert (NULL = plain)
};

namespace gs {

// ---- launch wrappers (each returns cudaGetLastError() of its launches) ----
cudaError_t launch_preprocess(gs_ctx* c, int n_views, const DevConst& k, cudaStream_t s);
cudaError_t launch_preprocess_backward(gs_ctx* c, const DevConst& k, bool add_reg, cudaStream_t s);
// Stable LSD radix sort of (u32 key, u32 value) pairs on the low `bits` bits.
// The count is min(*n_dev, n_max); n_hint (host estimate) only sizes the grid.
cudaError_t radix_sort_pairs(gs_ctx* c, uint32_t** keys, uint32_t** vals, const uint32_t* n_dev, uint32_t n_max,
                             uint32_t n_hint, int bits, int* out_buf, cudaStream_t s);
cudaError_t scan_tiles(gs_ctx* c, uint32_t n_max, const uint32_t* n_dev, cudaStream_t s);
cudaError_t emit_pairs(gs_ctx* c, uint32_t n_items, const uint32_t* n_dev, cudaStream_t s);
// exclusive scan of n u32 values (in may equal out); the total goes to *total_dev
cudaError_t scan_u32(gs_ctx* c, const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total_dev, cudaStream_t s);
cudaError_t compute_ranges(gs_ctx* c, cudaStream_t s);
// deterministic mode: per-item fixed-order sum of the pair gradient slots into grad2d
cudaError_t reduce_pair_grads(gs_ctx* c, cudaStream_t s);
cudaError_t launch_raster_forward(gs_ctx* c, const DevConst& k, float* rgb, int32_t* argmax, cudaStream_t s);
cudaError_t launch_raster_backward(gs_ctx* c, const DevConst& k, const float* dLdC, cudaStream_t s);
cudaError_t launch_count_work(gs_ctx* c, const DevConst& k, unsigned long long* out, cudaStream_t s);
// forward + L1 loss + adjoint of every (view, tile) in one persistent launch; writes the image,
// the screen-space gradients and one photometric partial per CTA (at most max_grid CTAs)
cudaError_t launch_raster_fused(gs_ctx* c, const DevConst& k, const float* target, const float* const* target_slot,
                                float* rgb, float* partials, int max_grid, int* grid_out, cudaStream_t s);
// the fixed-order sum of the photometric partials and the projection's planar-term partials
cudaError_t launch_loss_tail(gs_ctx* c, const DevConst& k, const float* photo_partials, int n_photo,
                             float* loss_out, cudaStream_t s);
cudaError_t launch_loss(gs_ctx* c, const DevConst& k, const float* rgb, const float* target, float* loss_out,
                        cudaStream_t s);
cudaError_t launch_adam(gs_ctx* c, cudaStream_t s);
// 10 log10(1 / MSE) of img against ref (n floats each) into out[0] (device)
cudaError_t launch_psnr(gs_ctx* c, const float* img, const float* ref, size_t n, float* out, cudaStream_t s);
int psnr_scratch_doubles();
int ssim_blocks(int width, int height, int n_views);
cudaError_t launch_ssim_loss(gs_ctx* c, const DevConst& k, const float* rgb, const float* target,
                             const float* const* target_slot, float* partials, cudaStream_t s);

// Adam (bias-corrected) with one learning rate per parameter row.
struct AdamArgs {
    float lr[kParamRows];
    float b1, b2, eps;
};
AdamArgs adam_args(const gs_ctx* c);

// inv_bc1, inv_bc2: reciprocals of the bias corrections 1 - beta^t (rounded once from float64)
__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, float lr, const AdamArgs& a,
                                            float inv_bc1, float inv_bc2) {
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    const float mh = m * inv_bc1, vh = v * inv_bc2;
    p -= __fdividef(lr * mh, sqrtf(vh) + a.eps);   // denominator < 2^126: 2-ulp division
}

// Bias corrections of the next Adam step from device state (so that a graph
// replays correctly): pw = {beta1^t, beta2^t} (float64 running products) after
// t = st[4] completed steps; st[1] = pair-buffer overflow flag (step skipped).
// Thread 0 of every CTA reads them before taking a ticket (st[2]); the last
// CTA of the launch advances pw and t, so every CTA uses the same t + 1.
// sbc = {1 / (1 - beta1^(t+1)), 1 / (1 - beta2^(t+1)), 1 if the step is skipped}.
__device__ __forceinline__ void adam_bias_begin(const AdamArgs& a, const uint32_t* st, const double* pw,
                                                float* sbc, double* spw) {
    const double p1 = pw[0] * (double)a.b1, p2 = pw[1] * (double)a.b2;
    spw[0] = p1;
    spw[1] = p2;
    sbc[0] = (float)(1.0 / (1.0 - p1));
    sbc[1] = (float)(1.0 / (1.0 - p2));
    sbc[2] = st[1] != 0u ? 1.f : 0.f;
}
__device__ __forceinline__ void adam_bias_end(uint32_t* st, double* pw, const float* sbc, const double* spw,
                                              uint32_t n_ctas) {
    if (atomicAdd(st + 2, 1u) == n_ctas - 1u) {
        if (sbc[2] == 0.f) {
            pw[0] = spw[0];
            pw[1] = spw[1];
            st[4] += 1u;
        }
        st[2] = 0u;
    }
}
cudaError_t launch_copy_T(gs_ctx* c, float* T_out, cudaStream_t s);
// learned initialiser (k_mlp.cu): overwrite the staged plain parameters of the points
cudaError_t mlp_initialise(gs_mlp* M, const DevCamera& cam, const float* image, const float* pts, int n, float* stage,
                           float* feat_tmp, cudaStream_t s);
// map management (k_map.cu)
cudaError_t launch_init_points(gs_ctx* c, const float* pts, const float* rgb, int n, const float* ref, int ref_stride,
                               int n_ref, int ref_is_self, float* out_params, int out_stride, cudaStream_t s);
cudaError_t launch_points_planar(const float* pts, int n, float* out, cudaStream_t s);
cudaError_t launch_insert_test(gs_ctx* c, const DevCamera& cam, const float* pts, int n, const float* image,
                               uint32_t* keep, float* stage, cudaStream_t s);
cudaError_t launch_append(gs_ctx* c, const float* stage, int n_stage, const uint32_t* keep, const uint32_t* pos,
                          cudaStream_t s);
cudaError_t launch_count_dominant(gs_ctx* c, const int32_t* argmax, size_t n_pix, cudaStream_t s);
cudaError_t launch_split_flags(gs_ctx* c, uint32_t* flags, cudaStream_t s);
cudaError_t launch_split_scatter(gs_ctx* c, const uint32_t* flags, const uint32_t* pos, uint32_t n_split,
                                 const float* normals, float* P2, float* M2, float* V2, cudaStream_t s);

}  // namespace gs
