// C ABI and host runtime: context, buffers, the render / loss / backward /
// step sequence, and the CUDA-graph mapping iteration.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "gs_internal.cuh"

using namespace gs;

namespace {

int fail(gs_ctx* c, int code, const char* what, cudaError_t e = cudaSuccess) {
    // the error is reported here; clear the runtime's last-error slot so that a
    // later cudaGetLastError() check does not see it again
    if (e != cudaSuccess) cudaGetLastError();
    char buf[512];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", what);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return fail(c, GS_ERR_CUDA, #call, e_); \
    } while (0)

struct CamBatch {
    DevCamera cam[GS_MAX_VIEWS];
    int n;
    const float* target;   // the iteration's target image (read through the context's target slot)
};

__global__ void k_set_cams(CamBatch b, DevCamera* dst, const float** target_slot) {
    int i = threadIdx.x;
    if (i == 0 && target_slot != nullptr) *target_slot = b.target;
    if (i < b.n) dst[i] = b.cam[i];
}

__global__ void k_fill(float* p, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

DevConst dev_const(const gs_config& f) {
    DevConst k;
    k.near_z = f.near_z;
    k.dilation = f.dilation;
    k.lambda_floor = f.lambda_floor;
    k.radius_sigma = f.radius_sigma;
    k.alpha_min = f.alpha_min;
    k.alpha_max = f.alpha_max;
    k.T_min = f.T_min;
    k.lambda_color = f.lambda_color;
    k.lambda_reg = f.lambda_reg;
    k.reg_floor = f.reg_floor;
    return k;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

int ceil_log2(uint32_t x) {
    int b = 0;
    while ((1u << b) < x) ++b;
    return b;
}

bool camera_ok(const gs_camera& g, const gs_config& f) {
    if (g.width <= 0 || g.height <= 0 || g.width > f.max_width || g.height > f.max_height) return false;
    if (!(g.fx > 0.f) || !(g.fy > 0.f)) return false;
    const float* v[4] = {&g.fx, &g.fy, &g.cx, &g.cy};
    for (auto x : v)
        if (!std::isfinite(*x)) return false;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(g.R[i])) return false;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(g.t[i])) return false;
    return true;
}

void make_cam(const gs_camera& g, const gs_config& f, int tile, int view, DevCamera& d) {
    memcpy(d.R, g.R, sizeof(d.R));
    memcpy(d.t, g.t, sizeof(d.t));
    d.fx = g.fx;
    d.fy = g.fy;
    d.cx = g.cx;
    d.cy = g.cy;
    d.lim_x = f.fov_clamp * (0.5f * (float)g.width / g.fx);
    d.lim_y = f.fov_clamp * (0.5f * (float)g.height / g.fy);
    d.width = g.width;
    d.height = g.height;
    d.tiles_x = (g.width + tile - 1) / tile;
    d.tiles_y = (g.height + tile - 1) / tile;
    d.bin_base = view * d.tiles_x * d.tiles_y;
    d.pad = 0;
}

void free_pairs(gs_ctx* c) {
    for (int i = 0; i < 2; ++i) {
        cudaFree(c->pkey[i]);
        cudaFree(c->pval[i]);
        c->pkey[i] = c->pval[i] = nullptr;
    }
    cudaFree(c->emit_item);
    cudaFree(c->pairgrad);
    c->emit_item = nullptr;
    c->pairgrad = nullptr;
}

cudaError_t alloc_pairs(gs_ctx* c, int64_t cap) {
    free_pairs(c);
    c->pair_cap = cap;
    cudaError_t e;
    for (int i = 0; i < 2; ++i) {
        if ((e = dalloc(&c->pkey[i], (size_t)cap)) != cudaSuccess) return e;
        if ((e = dalloc(&c->pval[i], (size_t)cap)) != cudaSuccess) return e;
    }
    if (c->cfg.deterministic) {
        if ((e = dalloc(&c->emit_item, (size_t)cap)) != cudaSuccess) return e;
        if ((e = dalloc(&c->pairgrad, (size_t)cap * kPairGradStride)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void drop_graph(gs_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_src) cudaGraphDestroy(c->graph_src);
    c->graph = nullptr;
    c->graph_src = nullptr;
    c->graph_pending = false;
    c->graph_tnodes.clear();
    c->cam_node = nullptr;
}

const gs_ctx::Tuned* find_tuned(const gs_ctx* c, int w, int h, int views) {
    const int nb = ceil_log2((uint32_t)std::max(c->n, 1));
    for (const auto& t : c->tuned)
        if (t.w == w && t.h == h && t.views == views && t.nb == nb) return &t;
    return nullptr;
}

// Tile size and pixels per thread of a render: the autotuner's candidate while
// it times one, else the configured values, else the tuned choice, else 16 / 1.
void pick_layout(gs_ctx* c, int w, int h, int views, int& tile, int& ppt) {
    if (c->cfg.deterministic) {   // one warp per tile: no ordering question inside a CTA
        tile = 8;
        ppt = 2;
        return;
    }
    if (c->force_tile) {
        tile = c->force_tile;
        ppt = c->force_ppt;
        return;
    }
    const gs_ctx::Tuned* t = c->cfg.tile_size == 0 ? find_tuned(c, w, h, views) : nullptr;
    tile = c->cfg.tile_size == 8 || c->cfg.tile_size == 16 ? c->cfg.tile_size : (t ? t->tile : 16);
    const int want = c->cfg.pixels_per_thread;
    if (want == 1 || want == 2 || (want == 4 && tile == 16))
        ppt = want;
    else
        ppt = (t && t->tile == tile) ? t->ppt : 1;
}

// Set up the per-view cameras of a render and upload them with a kernel (no
// host-memory copy, so the same sequence can be captured into a graph).
int prepare_views(gs_ctx* c, const gs_camera* cams, int n_views, CamBatch& b) {
    if (n_views < 1 || n_views > c->cfg.max_views) return fail(c, GS_ERR_ARG, "n_views out of range");
    if (cams == nullptr) return fail(c, GS_ERR_ARG, "cams is NULL");
    for (int v = 0; v < n_views; ++v) {
        if (!camera_ok(cams[v], c->cfg)) return fail(c, GS_ERR_ARG, "invalid camera");
        if (cams[v].width != cams[0].width || cams[v].height != cams[0].height)
            return fail(c, GS_ERR_ARG, "all views of one call must share one image size");
    }
    int tile = 16, ppt = 1;
    pick_layout(c, cams[0].width, cams[0].height, n_views, tile, ppt);
    memset(&b, 0, sizeof(b));
    b.n = n_views;
    for (int v = 0; v < n_views; ++v) make_cam(cams[v], c->cfg, tile, v, b.cam[v]);
    int bins = n_views * b.cam[0].tiles_x * b.cam[0].tiles_y;
    if (bins > c->max_bins) return fail(c, GS_ERR_ARG, "too many tiles for the configured maximum image size");
    c->tile = tile;
    c->n_views = n_views;
    c->width = cams[0].width;
    c->height = cams[0].height;
    c->n_bins = bins;
    c->ppt = ppt;
    memcpy(c->hcam, b.cam, sizeof(DevCamera) * n_views);
    return GS_OK;
}

int setup_views(gs_ctx* c, const gs_camera* cams, int n_views, cudaStream_t s) {
    CamBatch b;
    int code = prepare_views(c, cams, n_views, b);
    if (code != GS_OK) return code;
    ++c->launches;
    k_set_cams<<<1, 32, 0, s>>>(b, c->dcam, c->target_slot);
    CK(cudaGetLastError());
    return GS_OK;
}

cudaEvent_t take_event(gs_ctx* c) {
    if (!c->tpool.empty()) {
        cudaEvent_t e = c->tpool.back();
        c->tpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records CUDA events around one phase on the launching stream when timing is on.
struct Phase {
    gs_ctx* c;
    cudaStream_t s;
    cudaEvent_t end = nullptr;
    Phase(gs_ctx* c_, int id, cudaStream_t s_) : c(c_), s(s_) {
        if (!(c->timing & (1u << id))) return;
        cudaEvent_t a = take_event(c);
        end = take_event(c);
        if (!a || !end) {
            end = nullptr;
            return;
        }
        if (c->capturing) {
            // captured as an event-record node; each replay is given fresh events
            cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
            c->cap_phases.push_back({id, a, end});
        } else {
            cudaEventRecord(a, s);
            c->trec.push_back({id, a, end});
        }
    }
    ~Phase() {
        if (!end) return;
        if (c->capturing)
            cudaEventRecordWithFlags(end, s, cudaEventRecordExternal);
        else
            cudaEventRecord(end, s);
    }
};

// A non-finite loss or gradient of an earlier iteration (dcount[10], set by the loss total and
// by Adam, which leaves a parameter with a non-finite gradient unchanged) is reported once by
// the next call that reads the device flags, then cleared.
int check_nonfinite(gs_ctx* c, uint32_t flag, cudaStream_t s) {
    if (flag == 0u) return GS_OK;
    CK(cudaMemsetAsync(c->dcount + 10, 0, sizeof(uint32_t), s));
    c->hflags[10] = 0u;
    return fail(c, GS_ERR_NONFINITE,
                "an earlier iteration had a non-finite loss or gradient (parameters whose gradient was not "
                "finite were left unchanged)");
}

// The zeroing a mapping iteration needs before its pair emission (overflow flag, compositing
// work queues, bin ranges) and before its adjoint (screen gradients), issued on the side stream
// at the iteration's start so that it runs beside the projection and the depth sort; back_half
// and iteration_tail wait for it instead of zeroing on the main stream.
int side_begin(gs_ctx* c, cudaStream_t s) {
    CK(cudaEventRecord(c->side_ev[0], s));
    CK(cudaStreamWaitEvent(c->side, c->side_ev[0], 0));
    CK(cudaMemsetAsync(c->dcount + 1, 0, sizeof(uint32_t), c->side));
    CK(cudaMemsetAsync(c->dcount + 6, 0, 2 * sizeof(uint32_t), c->side));   // the compositing work queues
    CK(cudaMemsetAsync(c->ranges, 0, sizeof(uint2) * (size_t)c->n_bins, c->side));
    CK(cudaEventRecord(c->side_ev[1], c->side));   // (waited for before the pair emission)
    CK(cudaMemsetAsync(c->grad2d, 0, sizeof(float) * kGrad2dStride * c->n_views * (size_t)c->n, c->side));
    CK(cudaEventRecord(c->side_ev[2], c->side));
    c->side_zeroed = true;
    return GS_OK;
}

// An iteration that stopped part-way after side_begin (an error, or the report of a non-finite
// value): the side stream's zeroing is joined to s, and the other entry points zero on their own
// stream again. Returns `code`.
int side_abort(gs_ctx* c, cudaStream_t s, int code) {
    if (c->side_zeroed) {
        cudaEventRecord(c->side_ev[4], c->side);
        cudaStreamWaitEvent(s, c->side_ev[4], 0);
        c->side_zeroed = false;
    }
    return code;
}

// Projection, depth sort, scan. Leaves P in dcount[0].
int front_half(gs_ctx* c, const DevConst& k, cudaStream_t s) {
    const uint32_t items = (uint32_t)c->n_views * (uint32_t)c->n;
    Phase ph(c, GS_PHASE_PROJECT, s);
    CK(launch_preprocess(c, c->n_views, k, s));
    // the visible items, compacted in item order, sorted by depth (dcount[8] of them)
    int buf = 0;
    const uint32_t hint = c->visible_hint ? std::min(c->visible_hint + c->visible_hint / 4 + 256, items) : items;
    CK(radix_sort_pairs(c, c->dkey, c->dval, c->dcount + 8, items, hint, 32, &buf, s));
    CK(scan_tiles(c, items, c->dcount + 8, s));
    return GS_OK;
}

// Emission, bin sort, ranges, and (unless rgb is NULL) the forward raster.
int back_half(gs_ctx* c, const DevConst& k, float* rgb, int32_t* argmax, cudaStream_t s) {
    const uint32_t items = (uint32_t)c->n_views * (uint32_t)c->n;
    {
        Phase ph(c, GS_PHASE_BIN, s);
        if (c->side_zeroed)
            CK(cudaStreamWaitEvent(s, c->side_ev[1], 0));   // overflow flag and ranges zeroed
        else
            CK(cudaMemsetAsync(c->dcount + 1, 0, sizeof(uint32_t), s));
        CK(emit_pairs(c, items, c->dcount + 8, s));
        int bits = std::max(1, ceil_log2((uint32_t)c->n_bins));
        CK(radix_sort_pairs(c, c->pkey, c->pval, c->dcount, (uint32_t)std::min<int64_t>(c->pair_cap, 0xFFFFFFFFll),
                            c->pairs_hint, bits, &c->pair_buf, s));
        CK(compute_ranges(c, s));
    }
    if (!rgb) return GS_OK;
    Phase ph(c, GS_PHASE_RASTER_FWD, s);
    CK(launch_raster_forward(c, k, rgb, argmax, s));
    return GS_OK;
}

int render_empty(gs_ctx* c, float* rgb, float* T, int32_t* argmax, cudaStream_t s) {
    const size_t HW = (size_t)c->width * c->height;
    CK(cudaMemsetAsync(rgb, 0, sizeof(float) * 3 * HW * c->n_views, s));
    ++c->launches;
    k_fill<<<64, 256, 0, s>>>(c->T_final, HW * c->n_views, 1.f);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(c->n_last, 0, sizeof(uint32_t) * HW * c->n_views, s));
    if (argmax) CK(cudaMemsetAsync(argmax, 0xFF, sizeof(int32_t) * HW * c->n_views, s));
    CK(launch_copy_T(c, T, s));
    CK(cudaMemsetAsync(c->dcount, 0, sizeof(uint32_t), s));
    return GS_OK;
}

}  // namespace

extern "C" {

void gs_default_config(gs_config* f) {
    if (!f) return;
    memset(f, 0, sizeof(*f));
    f->near_z = 0.2f;
    f->fov_clamp = 1.3f;
    f->dilation = 0.3f;
    f->lambda_floor = 0.1f;
    f->radius_sigma = 3.f;
    f->alpha_min = 1.f / 255.f;
    f->alpha_max = 0.99f;
    f->T_min = 1e-4f;
    f->lambda_color = 1.f;
    f->lambda_reg = 1.f;
    f->reg_floor = 0.01f;
    f->lambda_photo = 0.f;
    f->beta1 = 0.9f;
    f->beta2 = 0.999f;
    f->eps = 1e-15f;
    f->lr[0] = 1e-3f;
    f->lr[1] = 5e-3f;
    f->lr[2] = 1e-3f;
    f->lr[3] = 5e-2f;
    f->lr[4] = 2.5e-3f;
    f->split_thresh = 2e-4f;
    f->split_factor = 1.6f;
    f->insert_opacity = 0.99f;
    f->tile_size = 16;
    f->capacity = 1 << 20;
    f->max_views = 8;
    f->max_width = 1280;
    f->max_height = 720;
    f->pair_capacity = 0;
    f->seed = 0x5eedULL;
    f->deterministic = 0;
}

int gs_create(const gs_config* cfg, int device, gs_ctx** out) {
    if (!cfg || !out) return GS_ERR_ARG;
    *out = nullptr;
    if (cfg->capacity <= 0 || cfg->max_views < 1 || cfg->max_views > GS_MAX_VIEWS || cfg->max_width <= 0 ||
        cfg->max_height <= 0 || (cfg->tile_size != 0 && cfg->tile_size != 8 && cfg->tile_size != 16) ||
        (cfg->pixels_per_thread != 0 && cfg->pixels_per_thread != 1 && cfg->pixels_per_thread != 2 &&
         cfg->pixels_per_thread != 4))
        return GS_ERR_ARG;
    if ((int64_t)cfg->capacity * cfg->max_views >= (int64_t)0xFFFFFFFF) return GS_ERR_ARG;
    if (!(cfg->lambda_photo >= 0.f && cfg->lambda_photo <= 1.f)) return GS_ERR_ARG;
    gs_ctx* c = new gs_ctx();
    c->cfg = *cfg;
    c->device = device;
    c->cap = (cfg->capacity + 3) & ~3;   // float4-aligned rows
    int code = GS_OK;
    do {
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) { code = fail(c, GS_ERR_CUDA, "cudaSetDevice", e); break; }
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
        if (c->num_sms <= 0) c->num_sms = 1;
        c->sort_blocks = c->num_sms * 4;
        c->n_partials = 2 * c->num_sms * 2;
        const size_t cap = (size_t)c->cap, V = (size_t)cfg->max_views;
        const size_t maxpix = (size_t)cfg->max_width * cfg->max_height;
        c->max_bins = (int)(V * ((cfg->max_width + 7) / 8) * ((cfg->max_height + 7) / 8));
        int64_t pc = cfg->pair_capacity > 0 ? cfg->pair_capacity : (int64_t)8 * cap * V;
        pc = std::min<int64_t>(pc, kMaxPairs);
        bool ok = true;
        ok = ok && dalloc(&c->params, kParamRows * cap) == cudaSuccess;
        ok = ok && dalloc(&c->grads, kParamRows * cap) == cudaSuccess;
        ok = ok && dalloc(&c->adam_m, kParamRows * cap) == cudaSuccess;
        ok = ok && dalloc(&c->adam_v, kParamRows * cap) == cudaSuccess;
        ok = ok && dalloc(&c->dens_sum, cap) == cudaSuccess;
        ok = ok && dalloc(&c->dens_cnt, cap) == cudaSuccess;
        ok = ok && dalloc(&c->dom_cnt, cap) == cudaSuccess;
        ok = ok && dalloc(&c->adam_pw, 2) == cudaSuccess;
        ok = ok && dalloc(&c->dcam, V) == cudaSuccess;
        ok = ok && dalloc(&c->rec, 3 * V * cap) == cudaSuccess;
        ok = ok && dalloc(&c->tiles_touched, V * cap) == cudaSuccess;
        ok = ok && dalloc(&c->depth, V * cap) == cudaSuccess;
        for (int i = 0; i < 2; ++i) {
            ok = ok && dalloc(&c->dkey[i], V * cap) == cudaSuccess;
            ok = ok && dalloc(&c->dval[i], V * cap) == cudaSuccess;
        }
        ok = ok && dalloc(&c->offsets, V * cap) == cudaSuccess;
        ok = ok && dalloc(&c->ranges, (size_t)c->max_bins) == cudaSuccess;
        ok = ok && dalloc(&c->work_order, (size_t)c->max_bins) == cudaSuccess;
        ok = ok && dalloc(&c->work_order_next, (size_t)c->max_bins) == cudaSuccess;
        ok = ok && dalloc(&c->work_order_graph, (size_t)c->max_bins) == cudaSuccess;
        ok = ok && dalloc(&c->T_final, V * maxpix) == cudaSuccess;
        ok = ok && dalloc(&c->n_last, V * maxpix) == cudaSuccess;
        ok = ok && dalloc(&c->dLdC, 3 * V * maxpix) == cudaSuccess;
        ok = ok && dalloc(&c->grad2d, kGrad2dStride * V * cap) == cudaSuccess;
        ok = ok && dalloc(&c->hist, (size_t)256 * c->sort_blocks + 256) == cudaSuccess;
        ok = ok && dalloc(&c->dcount, 16) == cudaSuccess;
        ok = ok && dalloc(&c->vis_blocks, V * ((cap + 255) / 256) + 1) == cudaSuccess;
        ok = ok && dalloc(&c->target_slot, 1) == cudaSuccess;
        if (cfg->lambda_photo > 0.f) {
            ok = ok && dalloc(&c->ssim_maps, (size_t)3 * 3 * V * maxpix) == cudaSuccess;
            ok = ok && dalloc(&c->ssim_part, (size_t)2 * ssim_blocks(cfg->max_width, cfg->max_height,
                                                                       cfg->max_views)) == cudaSuccess;
        }
        ok = ok && dalloc(&c->partials, (size_t)c->n_partials + 8) == cudaSuccess;
        ok = ok && dalloc(&c->psnr_part, (size_t)psnr_scratch_doubles()) == cudaSuccess;
        ok = ok && dalloc(&c->reg_part, (cap + 255) / 256 + 1) == cudaSuccess;
        if (cfg->deterministic) ok = ok && dalloc(&c->tile_part, (size_t)c->max_bins) == cudaSuccess;
        c->n_fpart = 32 * c->num_sms;   // at most 32 resident CTAs per SM
        ok = ok && dalloc(&c->fpart, (size_t)c->n_fpart) == cudaSuccess;
        ok = ok && alloc_pairs(c, pc) == cudaSuccess;
        ok = ok && cudaMallocHost((void**)&c->hcount, sizeof(uint32_t) * 16) == cudaSuccess;
        ok = ok && cudaMallocHost((void**)&c->hflags, sizeof(uint32_t) * 16) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 6; ++i)
            ok = ok && cudaEventCreateWithFlags(&c->side_ev[i], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&c->graph_done, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 2; ++i)
            for (cudaEvent_t* ev : {&c->h2d_start[i], &c->h2d_ready[i], &c->h2d_free[i]})
                ok = ok && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) { code = fail(c, GS_ERR_OOM, "device allocation failed"); break; }
        uint32_t init[16] = {0, 0, 0, 0xFFFFFFFFu, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        e = cudaMemcpy(c->dcount, init, sizeof(init), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(c->adam_m, 0, sizeof(float) * kParamRows * cap);
        if (e == cudaSuccess) e = cudaMemset(c->adam_v, 0, sizeof(float) * kParamRows * cap);
        if (e == cudaSuccess) e = cudaMemset(c->grads, 0, sizeof(float) * kParamRows * cap);
        if (e == cudaSuccess) e = cudaMemset(c->grad2d, 0, sizeof(float) * kGrad2dStride * V * cap);
        if (e == cudaSuccess) e = cudaMemset(c->dens_sum, 0, sizeof(float) * cap);
        if (e == cudaSuccess) e = cudaMemset(c->dens_cnt, 0, sizeof(float) * cap);
        if (e == cudaSuccess) e = cudaMemset(c->dom_cnt, 0, sizeof(uint32_t) * cap);
        const double pw1[2] = {1.0, 1.0};
        if (e == cudaSuccess) e = cudaMemcpy(c->adam_pw, pw1, sizeof(pw1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { code = fail(c, GS_ERR_CUDA, "initialisation", e); break; }
    } while (0);
    if (code != GS_OK) {
        gs_destroy(c);
        return code;
    }
    *out = c;
    return GS_OK;
}

void gs_destroy(gs_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    drop_graph(c);
    for (auto& r : c->trec) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->tpool) cudaEventDestroy(e);
    void* ptrs[] = {c->params, c->grads, c->adam_m, c->adam_v, c->dens_sum, c->dens_cnt, c->dom_cnt, c->adam_pw, c->dcam, c->rec,
                    c->tiles_touched, c->depth, c->dkey[0], c->dkey[1], c->dval[0], c->dval[1], c->offsets, c->ranges,
                    c->work_order, c->work_order_next, c->work_order_graph, c->T_final, c->n_last, c->dLdC, c->grad2d, c->hist, c->vis_blocks, (void*)c->target_slot, c->ssim_maps, c->ssim_part, c->dcount,
                    c->partials, c->psnr_part, c->reg_part, c->tile_part, c->fpart,
                    c->own_rgb, c->tgt_stage[0], c->tgt_stage[1]};
    for (void* p : ptrs) cudaFree(p);
    free_pairs(c);
    if (c->hcount) cudaFreeHost(c->hcount);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) cudaStreamDestroy(c->side);
    for (int i = 0; i < 6; ++i)
        if (c->side_ev[i]) cudaEventDestroy(c->side_ev[i]);
    if (c->graph_done) cudaEventDestroy(c->graph_done);
    if (c->copy) cudaStreamDestroy(c->copy);
    for (int i = 0; i < 2; ++i)
        for (cudaEvent_t ev : {c->h2d_start[i], c->h2d_ready[i], c->h2d_free[i]})
            if (ev) cudaEventDestroy(ev);
    delete c;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->err.c_str() : "null context"; }

int gs_num_gaussians(const gs_ctx* c) { return c ? c->n : 0; }

int gs_tile_size(const gs_ctx* c) { return c ? c->tile : 0; }

int gs_pixels_per_thread(const gs_ctx* c) { return c ? c->ppt : 0; }

int64_t gs_launch_count(const gs_ctx* c) { return c ? c->launches : 0; }

int gs_set_params(gs_ctx* c, const float* params_dev, int n, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (n < 0 || (n > 0 && !params_dev)) return fail(c, GS_ERR_ARG, "bad params");
    if (n > c->cap) return fail(c, GS_ERR_CAPACITY, "more Gaussians than the configured capacity");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    if (n > 0)
        CK(cudaMemcpy2DAsync(c->params, sizeof(float) * c->cap, params_dev, sizeof(float) * n, sizeof(float) * n,
                             kParamRows, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(c->adam_m, 0, sizeof(float) * kParamRows * c->cap, s));
    CK(cudaMemsetAsync(c->adam_v, 0, sizeof(float) * kParamRows * c->cap, s));
    CK(cudaMemsetAsync(c->dens_sum, 0, sizeof(float) * c->cap, s));
    CK(cudaMemsetAsync(c->dens_cnt, 0, sizeof(float) * c->cap, s));
    CK(cudaMemsetAsync(c->dom_cnt, 0, sizeof(uint32_t) * c->cap, s));
    CK(cudaMemsetAsync(c->dcount + 4, 0, sizeof(uint32_t), s));
    {
        static const double pw1[2] = {1.0, 1.0};
        CK(cudaMemcpyAsync(c->adam_pw, pw1, sizeof(pw1), cudaMemcpyHostToDevice, s));
    }
    c->n = n;
    c->adam_t = 0;
    c->n_views = 0;
    c->loss_ready = c->backward_ready = false;
    drop_graph(c);
    return GS_OK;
}

int gs_get_params(gs_ctx* c, float* out, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (c->n == 0) return GS_OK;
    if (!out) return fail(c, GS_ERR_ARG, "out is NULL");
    CK(cudaMemcpy2DAsync(out, sizeof(float) * c->n, c->params, sizeof(float) * c->cap, sizeof(float) * c->n,
                         kParamRows, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return GS_OK;
}

int gs_get_grads(gs_ctx* c, float* out, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (c->n == 0) return GS_OK;
    if (!out) return fail(c, GS_ERR_ARG, "out is NULL");
    CK(cudaMemcpy2DAsync(out, sizeof(float) * c->n, c->grads, sizeof(float) * c->cap, sizeof(float) * c->n,
                         kParamRows, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return GS_OK;
}

int gs_set_grads(gs_ctx* c, const float* in, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (c->n == 0) return GS_OK;
    if (!in) return fail(c, GS_ERR_ARG, "grads_dev is NULL");
    CK(cudaMemcpy2DAsync(c->grads, sizeof(float) * c->cap, in, sizeof(float) * c->n, sizeof(float) * c->n,
                         kParamRows, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return GS_OK;
}

int gs_render(gs_ctx* c, const gs_camera* cams, int n_views, float* rgb, float* T, int32_t* argmax, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!rgb) return fail(c, GS_ERR_ARG, "rgb_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    c->loss_ready = c->backward_ready = false;
    int code = setup_views(c, cams, n_views, s);
    if (code != GS_OK) {
        c->n_views = 0;
        return code;
    }
    const DevConst k = dev_const(c->cfg);
    c->rendered_rgb = rgb;
    if (c->n == 0) return render_empty(c, rgb, T, argmax, s);
    if ((code = front_half(c, k, s)) != GS_OK) {
        c->n_views = 0;   // no image to take a loss of
        return code;
    }
    // size the pair buffers: read P back (the one synchronisation of a render)
    CK(cudaMemcpyAsync(c->hcount, c->dcount, sizeof(uint32_t) * 11, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((code = check_nonfinite(c, c->hcount[10], s)) != GS_OK) {
        c->n_views = 0;
        return code;
    }
    const int64_t P = c->hcount[0];
    c->visible_hint = c->hcount[8];
    c->pairs_hint = (uint32_t)std::min<int64_t>(P, 0xFFFFFFFFll);
    if (P > c->pair_cap) {
        drop_graph(c);
        if (alloc_pairs(c, std::min<int64_t>(P + P / 2 + 1024, kMaxPairs)) != cudaSuccess) {
            c->n_views = 0;
            return fail(c, GS_ERR_OOM, "growing the pair buffers failed");
        }
        if (P > c->pair_cap) {
            c->n_views = 0;
            return fail(c, GS_ERR_CAPACITY, "pair count exceeds 2^32");
        }
    }
    if ((code = back_half(c, k, rgb, argmax, s)) != GS_OK) {
        c->n_views = 0;
        return code;
    }
    CK(launch_copy_T(c, T, s));
    return GS_OK;
}

int gs_loss(gs_ctx* c, const float* target, float* loss_dev, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (c->n_views == 0 || !c->rendered_rgb) return fail(c, GS_ERR_STATE, "gs_loss before gs_render");
    if (!target) return fail(c, GS_ERR_ARG, "target_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    float* out = loss_dev ? loss_dev : c->partials + c->n_partials;
    const DevConst k = dev_const(c->cfg);
    Phase ph(c, GS_PHASE_LOSS, s);
    if (c->cfg.lambda_photo > 0.f) {
        CK(launch_ssim_loss(c, k, c->rendered_rgb, target, nullptr, c->ssim_part, s));
        CK(launch_loss_tail(c, k, c->ssim_part, 2 * ssim_blocks(c->width, c->height, c->n_views), out, s));
    } else {
        CK(launch_loss(c, k, c->rendered_rgb, target, out, s));
    }
    c->loss_ready = true;
    return GS_OK;
}

int gs_backward(gs_ctx* c, const float* dL_drgb, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (c->n_views == 0) return fail(c, GS_ERR_STATE, "gs_backward before gs_render");
    if (!dL_drgb && !c->loss_ready) return fail(c, GS_ERR_STATE, "gs_backward(NULL) before gs_loss");
    cudaStream_t s = (cudaStream_t)stream;
    const DevConst k = dev_const(c->cfg);
    if (c->n == 0) {
        c->backward_ready = true;
        return GS_OK;
    }
    CK(cudaMemsetAsync(c->grad2d, 0, sizeof(float) * kGrad2dStride * c->n_views * (size_t)c->n, s));
    {
        Phase ph(c, GS_PHASE_RASTER_BWD, s);
        CK(launch_raster_backward(c, k, dL_drgb ? dL_drgb : c->dLdC, s));
        CK(reduce_pair_grads(c, s));   // deterministic mode only
    }
    Phase ph(c, GS_PHASE_PROJECT_BWD, s);
    CK(launch_preprocess_backward(c, k, dL_drgb == nullptr, s));
    c->backward_ready = true;
    return GS_OK;
}

int gs_step(gs_ctx* c, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!c->backward_ready) return fail(c, GS_ERR_STATE, "gs_step before gs_backward");
    cudaStream_t s = (cudaStream_t)stream;
    Phase ph(c, GS_PHASE_ADAM, s);
    CK(launch_adam(c, s));
    c->adam_t += 1;
    c->backward_ready = false;
    return GS_OK;
}

// Everything of a mapping iteration after the projection and depth sort: binning,
// compositing + loss + adjoint (one fused kernel with pure L1; forward, SSIM loss and
// adjoint as three kernels with the SSIM term), the loss total, the projection adjoint
// and Adam. Shared by the direct first call of gs_iterate and its graph capture; a
// captured iteration also copies the device flags (pair count, overflow, non-finite values) to
// the host, where the next call reads them.
static int iteration_tail(gs_ctx* c, const DevConst& k, const float* target, const float* const* slot, float* rgb,
                          float* loss_out, bool capture, cudaStream_t s) {
    const bool ssim = c->cfg.lambda_photo > 0.f;
    int cc = back_half(c, k, ssim ? rgb : nullptr, nullptr, s);
    if (cc != GS_OK) return cc;
    if (ssim) {
        Phase ph(c, GS_PHASE_LOSS, s);
        if (launch_ssim_loss(c, k, rgb, target, slot, c->ssim_part, s) != cudaSuccess ||
            launch_loss_tail(c, k, c->ssim_part, 2 * ssim_blocks(c->width, c->height, c->n_views), loss_out, s) !=
                cudaSuccess)
            return fail(c, GS_ERR_CUDA, "loss launch", cudaGetLastError());
    }
    if (c->side_zeroed)
        CK(cudaStreamWaitEvent(s, c->side_ev[2], 0));   // work queues and grad2d zeroed
    else
        CK(cudaMemsetAsync(c->grad2d, 0, sizeof(float) * kGrad2dStride * c->n_views * (size_t)c->n, s));
    // the loss total (and, when capturing, the copy of the device flags: pair count, overflow,
    // non-finite values) on the side stream, beside the projection adjoint and Adam
    cudaStream_t ts = c->side_zeroed ? c->side : s;
    if (ssim) {
        Phase ph(c, GS_PHASE_RASTER_BWD, s);
        CK(launch_raster_backward(c, k, c->dLdC, s));
        if (c->side_zeroed) {
            CK(cudaEventRecord(c->side_ev[3], s));
            CK(cudaStreamWaitEvent(ts, c->side_ev[3], 0));
        }
    } else {
        int fgrid = 0;
        {
            Phase ph(c, GS_PHASE_RASTER_FUSED, s);
            CK(launch_raster_fused(c, k, target, slot, rgb, c->fpart, c->n_fpart, &fgrid, s));
        }
        if (c->side_zeroed) {
            CK(cudaEventRecord(c->side_ev[3], s));
            CK(cudaStreamWaitEvent(ts, c->side_ev[3], 0));
        }
        Phase ph(c, GS_PHASE_LOSS, ts);
        // the deterministic mode sums the per-tile partials, the default the per-CTA ones
        const bool det = c->tile_part != nullptr;
        CK(launch_loss_tail(c, k, det ? c->tile_part : c->fpart, det ? c->n_bins : fgrid, loss_out, ts));
    }
    if (capture) CK(cudaMemcpyAsync(c->hflags, c->dcount, sizeof(uint32_t) * 11, cudaMemcpyDeviceToHost, ts));
    if (c->order_ahead)   // the compositing is done with the current order: the next one goes in place
        CK(cudaMemcpyAsync(c->work_order, c->work_order_next, sizeof(uint32_t) * (size_t)c->n_bins,
                           cudaMemcpyDeviceToDevice, ts));
    {
        Phase ph(c, GS_PHASE_PROJECT_BWD, s);
        CK(reduce_pair_grads(c, s));
        CK(launch_preprocess_backward(c, k, true, s));
    }
    {
        Phase ph(c, GS_PHASE_ADAM, s);
        CK(launch_adam(c, s));
    }
    if (c->side_zeroed) {
        CK(cudaEventRecord(c->side_ev[4], ts));
        CK(cudaStreamWaitEvent(s, c->side_ev[4], 0));   // join: the iteration ends on s
        c->side_zeroed = false;
    }
    return GS_OK;
}

// The autotuner: for each (tile size, pixels per thread) candidate on the
// caller's views, one plain render sizes the pair buffers, then the part of the
// mapping iteration that depends on the layout (projection, binning, sort and
// the fused compositing + L1 + adjoint kernel) is timed; the fastest is kept
// for this (image size, views, N-bucket). The adjoint of the projection and
// Adam are left out, so the map and its statistics are unchanged.
static int autotune(gs_ctx* c, const gs_camera* cams, int n_views, const float* target, float* rgb,
                    cudaStream_t s) {
    static const int cand[][2] = {{16, 1}, {16, 2}, {16, 4}, {8, 1}, {8, 2}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const uint32_t timing = c->timing;
    c->timing = 0;
    float best = 1e30f;
    int bt = 16, bp = 1, code = GS_OK;
    for (const auto& cd : cand) {
        c->force_tile = cd[0];
        c->force_ppt = cd[1];
        float ms = 0.f;
        code = gs_render(c, cams, n_views, rgb, nullptr, nullptr, s);
        const DevConst k = dev_const(c->cfg);
        for (int rep = 0; rep < 2 && code == GS_OK; ++rep) {
            cudaEventRecord(e0, s);
            code = setup_views(c, cams, n_views, s);
            if (code == GS_OK) code = front_half(c, k, s);
            if (code == GS_OK) code = back_half(c, k, nullptr, nullptr, s);
            if (code == GS_OK &&
                cudaMemsetAsync(c->grad2d, 0, sizeof(float) * kGrad2dStride * c->n_views * (size_t)c->n, s) !=
                    cudaSuccess)
                code = GS_ERR_CUDA;
            int fgrid = 0;
            if (code == GS_OK &&
                launch_raster_fused(c, k, target, nullptr, rgb, c->fpart, c->n_fpart, &fgrid, s) != cudaSuccess)
                code = GS_ERR_CUDA;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) code = GS_ERR_CUDA;
            if (rep == 1) cudaEventElapsedTime(&ms, e0, e1);
        }
        if (code != GS_OK) break;
        if (ms < best) {
            best = ms;
            bt = cd[0];
            bp = cd[1];
        }
    }
    c->force_tile = c->force_ppt = 0;
    c->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (code != GS_OK) return code;
    c->tuned.push_back({cams[0].width, cams[0].height, n_views, ceil_log2((uint32_t)std::max(c->n, 1)), bt, bp});
    c->backward_ready = false;
    return GS_OK;
}

// The mapping iteration (gs_iterate without the argument checks).
static int iterate_core(gs_ctx* c, const gs_camera* cams, int n_views, const float* target, float* loss_dev,
                        float* rgb, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n_views < 1 || n_views > c->cfg.max_views || !cams) return fail(c, GS_ERR_ARG, "bad views");
    if (!rgb) {
        size_t need = (size_t)n_views * 3 * cams[0].width * cams[0].height;
        if (need > c->own_rgb_elems) {
            drop_graph(c);
            cudaFree(c->own_rgb);
            c->own_rgb = nullptr;
            c->own_rgb_elems = 0;
            if (dalloc(&c->own_rgb, need) != cudaSuccess) return fail(c, GS_ERR_OOM, "image buffer");
            c->own_rgb_elems = need;
        }
        rgb = c->own_rgb;
    }
    float* loss_out = loss_dev ? loss_dev : c->partials + c->n_partials;
    if (c->cfg.tile_size == 0 && !c->cfg.deterministic && c->n > 0 &&
        !find_tuned(c, cams[0].width, cams[0].height, n_views)) {
        if (n_views < 1 || n_views > c->cfg.max_views) return fail(c, GS_ERR_ARG, "bad views");
        drop_graph(c);
        int code = autotune(c, cams, n_views, target, rgb, s);
        if (code != GS_OK) return code;
    }
    // The flags of an earlier replay: a pair-buffer overflow there skipped its Adam step.
    if (c->graph && c->graph_pending && cudaEventQuery(c->graph_done) == cudaSuccess) {
        c->graph_pending = false;
        const uint32_t P = c->hflags[0];
        if (c->hflags[10] != 0u) return check_nonfinite(c, c->hflags[10], s);
        if (c->hflags[1] != 0u) {
            drop_graph(c);
            if (alloc_pairs(c, std::min<int64_t>((int64_t)P + P / 2 + 4096, kMaxPairs)) != cudaSuccess)
                return fail(c, GS_ERR_OOM, "growing the pair buffers failed");
            return fail(c, GS_ERR_CAPACITY, "an earlier iteration overflowed the pair buffer and skipped its update; "
                                            "the buffer has grown");
        }
        c->pairs_hint = P;
    }
    CamBatch b;
    int code = prepare_views(c, cams, n_views, b);
    if (code != GS_OK) return code;
    const bool same = c->graph && c->graph_views == n_views && c->graph_w == cams[0].width &&
                      c->graph_h == cams[0].height && c->graph_n == c->n && c->graph_tile == c->tile &&
                      c->graph_ppt == c->ppt && c->graph_pair_cap == c->pair_cap &&
                      c->graph_loss == loss_out && c->graph_rgb == rgb && c->graph_timing == c->timing;
    if (same) {
        // replay: new cameras go in as the upload kernel's parameters
        DevCamera* dst = c->dcam;
        const float** slot = c->target_slot;
        b.target = target;   // the graph reads the target through the slot: any buffer per call
        void* args[3] = {&b, &dst, &slot};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)k_set_cams;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        CK(cudaGraphExecKernelNodeSetParams(c->graph, c->cam_node, &kp));
        if (c->timing) {
            for (auto& tn : c->graph_tnodes) {
                cudaEvent_t ea = take_event(c), eb = take_event(c);
                CK(cudaGraphExecEventRecordNodeSetEvent(c->graph, tn.a, ea));
                CK(cudaGraphExecEventRecordNodeSetEvent(c->graph, tn.b, eb));
                c->trec.push_back({tn.phase, ea, eb});
            }
        }
        CK(cudaGraphLaunch(c->graph, s));
        CK(cudaEventRecord(c->graph_done, s));
        c->graph_pending = true;
        c->launches += c->graph_kernels;
        c->adam_t += 1;
        c->loss_ready = false;      // the fused kernel keeps dL/dC in registers
        c->backward_ready = false;
        c->rendered_rgb = rgb;
        return GS_OK;
    }
    // First iteration of this shape: the same kernels as a replay, run directly with one
    // synchronisation after the projection that sizes the pair buffers; then the whole
    // iteration is recorded into a graph for the following calls.
    drop_graph(c);
    if (c->n == 0) {
        code = gs_render(c, cams, n_views, rgb, nullptr, nullptr, stream);
        if (code == GS_OK) code = gs_loss(c, target, loss_dev, stream);
        if (code == GS_OK) code = gs_backward(c, nullptr, stream);
        if (code == GS_OK) code = gs_step(c, s);
        return code;
    }
    const DevConst k = dev_const(c->cfg);
    c->loss_ready = c->backward_ready = false;
    b.target = target;
    ++c->launches;
    k_set_cams<<<1, 32, 0, s>>>(b, c->dcam, c->target_slot);
    CK(cudaGetLastError());
    auto direct = [&]() -> int {
        int cd;
        if ((cd = side_begin(c, s)) != GS_OK) return cd;
        if ((cd = front_half(c, k, s)) != GS_OK) return cd;
        CK(cudaMemcpyAsync(c->hcount, c->dcount, sizeof(uint32_t) * 11, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if ((cd = check_nonfinite(c, c->hcount[10], s)) != GS_OK) return cd;
        const int64_t P = c->hcount[0];
        c->visible_hint = c->hcount[8];
        c->pairs_hint = (uint32_t)std::min<int64_t>(P, 0xFFFFFFFFll);
        // headroom for the replays' changing cameras
        const int64_t want = std::min<int64_t>(P + P / 4 + 4096, kMaxPairs);
        if (P > kMaxPairs) return fail(c, GS_ERR_CAPACITY, "pair count exceeds 2^32");
        if (want > c->pair_cap && alloc_pairs(c, want) != cudaSuccess)
            return fail(c, GS_ERR_OOM, "growing the pair buffers failed");
        return iteration_tail(c, k, target, c->target_slot, rgb, loss_out, false, s);
    };
    code = direct();
    if (code != GS_OK) return side_abort(c, s, code);
    c->adam_t += 1;
    c->rendered_rgb = rgb;
    const int64_t launches0 = c->launches;
    // the first replay composites in the order this direct call computed for the shape
    CK(cudaMemcpyAsync(c->work_order_graph, c->work_order, sizeof(uint32_t) * (size_t)c->n_bins,
                       cudaMemcpyDeviceToDevice, s));
    c->cap_phases.clear();
    c->capturing = true;
    cudaStream_t cs = c->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->capturing = false;
        return fail(c, GS_ERR_CUDA, "cudaStreamBeginCapture", e);
    }
    int cc = GS_OK;
    {
        ++c->launches;
        k_set_cams<<<1, 32, 0, cs>>>(b, c->dcam, c->target_slot);
        cc = side_begin(c, cs);
        // the direct call above left this shape's work order in work_order_graph for the first
        // replay; every replay reads that buffer and writes the next order into it
        c->order_ahead = true;
        std::swap(c->work_order, c->work_order_graph);
        if (cc == GS_OK) cc = front_half(c, k, cs);
        if (cc == GS_OK) cc = iteration_tail(c, k, target, c->target_slot, rgb, loss_out, true, cs);
    }
    if (cc != GS_OK) side_abort(c, cs, cc);   // joined, so that the capture ends cleanly
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    c->capturing = false;
    c->side_zeroed = false;
    if (c->order_ahead) std::swap(c->work_order, c->work_order_graph);
    c->order_ahead = false;
    c->graph_kernels = c->launches - launches0;
    c->launches = launches0;
    if (cc != GS_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return fail(c, GS_ERR_CUDA, "capturing the mapping iteration failed", e);
    }
    // locate the camera-upload node and the phase event nodes
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    c->graph_tnodes.clear();
    std::vector<cudaGraphNode_t> ta(c->cap_phases.size(), nullptr), tb(c->cap_phases.size(), nullptr);
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        cudaGraphNodeGetType(nd, &ty);
        if (ty == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == (void*)k_set_cams) c->cam_node = nd;
        } else if (ty == cudaGraphNodeTypeEventRecord) {
            cudaEvent_t ev;
            if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
            for (size_t i = 0; i < c->cap_phases.size(); ++i) {
                if (c->cap_phases[i].a == ev) ta[i] = nd;
                if (c->cap_phases[i].b == ev) tb[i] = nd;
            }
        }
    }
    for (size_t i = 0; i < c->cap_phases.size(); ++i)
        if (ta[i] && tb[i]) c->graph_tnodes.push_back({c->cap_phases[i].phase, ta[i], tb[i]});
    e = c->cam_node ? cudaGraphInstantiate(&c->graph, g, 0) : cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        c->graph = nullptr;
        c->graph_tnodes.clear();
        c->cam_node = nullptr;
        return fail(c, GS_ERR_CUDA, "instantiating the mapping iteration graph failed", e);
    }
    c->graph_src = g;
    c->graph_views = n_views;
    c->graph_w = cams[0].width;
    c->graph_h = cams[0].height;
    c->graph_n = c->n;
    c->graph_tile = c->tile;
    c->graph_ppt = c->ppt;
    c->graph_pair_cap = c->pair_cap;
    c->graph_loss = loss_out;
    c->graph_rgb = rgb;
    c->graph_timing = c->timing;
    return GS_OK;
}

int gs_iterate(gs_ctx* c, const gs_camera* cams, int n_views, const float* target, float* loss_dev, float* rgb,
               void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!target) return fail(c, GS_ERR_ARG, "target_dev is NULL");
    CK(cudaSetDevice(c->device));
    return iterate_core(c, cams, n_views, target, loss_dev, rgb, stream);
}

int gs_iterate_host(gs_ctx* c, const gs_camera* cams, int n_views, const float* target_host, float* loss_host,
                    float* rgb, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!target_host) return fail(c, GS_ERR_ARG, "target_host is NULL");
    if (n_views < 1 || n_views > c->cfg.max_views || !cams) return fail(c, GS_ERR_ARG, "bad views");
    if (!camera_ok(cams[0], c->cfg)) return fail(c, GS_ERR_ARG, "invalid camera");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    const size_t elems = (size_t)n_views * 3 * cams[0].width * cams[0].height;
    if (elems > c->tgt_stage_elems) {
        CK(cudaStreamSynchronize(c->copy));
        for (int i = 0; i < 2; ++i) CK(cudaEventSynchronize(c->h2d_free[i]));   // the buffers' last readers
        for (int i = 0; i < 2; ++i) {
            cudaFree(c->tgt_stage[i]);
            c->tgt_stage[i] = nullptr;
        }
        c->tgt_stage_elems = 0;
        for (int i = 0; i < 2; ++i)
            if (dalloc(&c->tgt_stage[i], elems) != cudaSuccess) return fail(c, GS_ERR_OOM, "target buffers");
        c->tgt_stage_elems = elems;
    }
    // the upload starts once the previous call's iteration has started on its stream (with the
    // host ahead of the device it runs beside that iteration) and the one before, the last reader
    // of this buffer, is done; this call's iteration waits for it. Host-side stream waits only:
    // each resolves to the record made by the call named, so no wait can refer to later work.
    const int k = c->h2d_k;
    CK(cudaStreamWaitEvent(c->copy, c->h2d_start[k ^ 1], 0));
    CK(cudaStreamWaitEvent(c->copy, c->h2d_free[k], 0));
    CK(cudaMemcpyAsync(c->tgt_stage[k], target_host, sizeof(float) * elems, cudaMemcpyHostToDevice, c->copy));
    CK(cudaEventRecord(c->h2d_ready[k], c->copy));
    CK(cudaEventRecord(c->h2d_start[k], s));
    CK(cudaStreamWaitEvent(s, c->h2d_ready[k], 0));
    c->h2d_k = k ^ 1;
    const int code = iterate_core(c, cams, n_views, c->tgt_stage[k], nullptr, rgb, stream);
    CK(cudaEventRecord(c->h2d_free[k], s));
    if (code != GS_OK) return code;
    if (loss_host)
        CK(cudaMemcpyAsync(loss_host, c->partials + c->n_partials, sizeof(float) * 3, cudaMemcpyDeviceToHost, s));
    return GS_OK;
}

int gs_psnr(gs_ctx* c, const float* img_dev, const float* ref_dev, int64_t n, float* out_dev, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (n <= 0 || !img_dev || !ref_dev || !out_dev) return fail(c, GS_ERR_ARG, "gs_psnr: bad arguments");
    CK(cudaSetDevice(c->device));
    CK(launch_psnr(c, img_dev, ref_dev, (size_t)n, out_dev, (cudaStream_t)stream));
    return GS_OK;
}

int gs_timing_enable(gs_ctx* c, int enable) {
    if (!c) return GS_ERR_ARG;
    for (auto& r : c->trec) {
        c->tpool.push_back(r.a);
        c->tpool.push_back(r.b);
    }
    c->trec.clear();
    c->timing = enable != 0 ? (1u << GS_N_PHASES) - 1u : 0u;
    return GS_OK;
}

int gs_timing_phases(gs_ctx* c, uint32_t mask) {
    const int code = gs_timing_enable(c, 0);
    if (code != GS_OK) return code;
    c->timing = mask & ((1u << GS_N_PHASES) - 1u);
    return GS_OK;
}

int gs_timing_read(gs_ctx* c, float* ms, int32_t* counts) {
    if (!c || !ms) return GS_ERR_ARG;
    for (int i = 0; i < GS_N_PHASES; ++i) {
        ms[i] = 0.f;
        if (counts) counts[i] = 0;
    }
    int code = GS_OK;
    for (auto& r : c->trec) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) {
            code = fail(c, GS_ERR_CUDA, "timing event", e);
            break;
        }
        if (r.phase >= 0 && r.phase < GS_N_PHASES) {
            ms[r.phase] += t;
            if (counts) counts[r.phase] += 1;
        }
    }
    for (auto& r : c->trec) {
        c->tpool.push_back(r.a);
        c->tpool.push_back(r.b);
    }
    c->trec.clear();
    return code;
}

int gs_debug_projection(gs_ctx* c, int view, double* out) {
    if (!c || !out) return GS_ERR_ARG;
    if (c->n_views == 0 || view < 0 || view >= c->n_views) return fail(c, GS_ERR_STATE, "no such rendered view");
    const size_t n = (size_t)c->n;
    std::vector<float4> rec(3 * n);
    std::vector<uint32_t> tl(n);
    std::vector<float> dep(n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && n)
        e = cudaMemcpy(rec.data(), c->rec + 3 * n * view, sizeof(float4) * 3 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && n)
        e = cudaMemcpy(tl.data(), c->tiles_touched + n * view, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && n) e = cudaMemcpy(dep.data(), c->depth + n * view, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "debug copy", e);
    const double k1 = -0.5 * (double)kLog2e, k2 = -(double)kLog2e;
    for (size_t i = 0; i < n; ++i) {
        const float4 a = rec[3 * i], q = rec[3 * i + 1], col = rec[3 * i + 2];
        out[0 * n + i] = (double)a.x + (double)q.w;
        out[1 * n + i] = (double)a.y + (double)col.w;
        out[2 * n + i] = q.x / k1;
        out[3 * n + i] = q.y / k2;
        out[4 * n + i] = q.z / k1;
        out[5 * n + i] = dep[i];
        out[6 * n + i] = a.z;
        out[7 * n + i] = (double)tl[i];
        out[8 * n + i] = a.z >= 0.f ? 1.0 : 0.0;
    }
    return GS_OK;
}

int gs_debug_pairs(gs_ctx* c, uint32_t* bins, uint32_t* vals, int64_t max, int64_t* count) {
    if (!c || !count) return GS_ERR_ARG;
    CK(cudaDeviceSynchronize());
    uint32_t P = 0;
    CK(cudaMemcpy(&P, c->dcount, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    *count = P;
    int64_t m = std::min<int64_t>(P, max);
    if (m > 0 && bins) CK(cudaMemcpy(bins, c->pkey[c->pair_buf], sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
    if (m > 0 && vals) {
        CK(cudaMemcpy(vals, c->pval[c->pair_buf], sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
        if (c->emit_item) {   // deterministic mode: the sorted values are emission indices
            std::vector<uint32_t> items((size_t)std::min<int64_t>(P, c->pair_cap));
            if (!items.empty())
                CK(cudaMemcpy(items.data(), c->emit_item, sizeof(uint32_t) * items.size(), cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < m; ++i) vals[i] = vals[i] < items.size() ? items[vals[i]] : 0xFFFFFFFFu;
        }
    }
    return GS_OK;
}

int gs_debug_work(gs_ctx* c, int64_t* out) {
    if (!c || !out) return GS_ERR_ARG;
    if (c->n_views == 0) return fail(c, GS_ERR_STATE, "no render");
    unsigned long long* d = nullptr;
    CK(cudaMalloc((void**)&d, sizeof(unsigned long long) * 4));
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemset(d, 0, sizeof(h));
    if (e == cudaSuccess && c->n > 0) e = launch_count_work(c, dev_const(c->cfg), d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    uint32_t P = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&P, c->dcount, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "work count", e);
    out[0] = c->n > 0 ? (int64_t)P : 0;
    out[1] = (int64_t)h[0];
    out[2] = (int64_t)h[1];
    out[3] = (int64_t)h[2];
    return GS_OK;
}

int gs_debug_grad2d(gs_ctx* c, float* out) {
    if (!c || !out) return GS_ERR_ARG;
    if (c->n_views == 0) return fail(c, GS_ERR_STATE, "no render");
    const size_t n = (size_t)c->n, items = n * c->n_views;
    float* g = (float*)malloc(sizeof(float) * kGrad2dStride * items);
    if (!g) return fail(c, GS_ERR_OOM, "host buffer");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(g, c->grad2d, sizeof(float) * kGrad2dStride * items, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free(g);
        return fail(c, GS_ERR_CUDA, "debug copy", e);
    }
    // the records hold the first five values without the factor ln 2 of d 2^p / dp; the exp2
    // scaling of the conic (a' = -a log2(e) / 2, b' = -b log2(e)) cancels it for a, b, c
    for (int v = 0; v < c->n_views; ++v)
        for (size_t i = 0; i < n; ++i) {
            const float* r = g + (v * n + i) * kGrad2dStride;
            float* o = out + (size_t)v * 9 * n;
            o[0 * n + i] = r[0] * kLn2;
            o[1 * n + i] = r[1] * kLn2;
            o[2 * n + i] = r[2] * -0.5f;
            o[3 * n + i] = -r[3];
            o[4 * n + i] = r[4] * -0.5f;
            o[5 * n + i] = r[5];
            o[6 * n + i] = r[6];
            o[7 * n + i] = r[7];
            o[8 * n + i] = r[8];
        }
    free(g);
    return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- map management

namespace {

struct Temp {
    void* p[8] = {nullptr};
    int k = 0;
    template <typename T>
    bool get(T** out, size_t count) {
        if (cudaMalloc((void**)out, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
            *out = nullptr;
            return false;
        }
        p[k++] = *out;
        return true;
    }
    ~Temp() {
        for (int i = 0; i < k; ++i) cudaFree(p[i]);
    }
};

void invalidate_render(gs_ctx* c) {
    c->n_views = 0;
    c->loss_ready = c->backward_ready = false;
    drop_graph(c);
}

}  // namespace

extern "C" {

int gs_init_map(gs_ctx* c, const float* pts, const float* rgb, int n, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (n < 0 || (n > 0 && (!pts || !rgb))) return fail(c, GS_ERR_ARG, "bad points");
    if ((int64_t)c->n + n > c->cap) return fail(c, GS_ERR_CAPACITY, "more Gaussians than the configured capacity");
    if (n == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    Temp t;
    float *ref = nullptr, *stage = nullptr;
    if (!t.get(&ref, 3 * (size_t)n) || !t.get(&stage, kParamRows * (size_t)n))
        return fail(c, GS_ERR_OOM, "temporary buffers");
    CK(launch_points_planar(pts, n, ref, s));
    CK(launch_init_points(c, pts, rgb, n, ref, n, n, 1, stage, n, s));
    CK(cudaMemcpy2DAsync(c->params + c->n, sizeof(float) * c->cap, stage, sizeof(float) * n, sizeof(float) * n,
                         kParamRows, cudaMemcpyDeviceToDevice, s));
    for (float* a : {c->adam_m, c->adam_v})
        CK(cudaMemset2DAsync(a + c->n, sizeof(float) * c->cap, 0, sizeof(float) * n, kParamRows, s));
    CK(cudaMemsetAsync(c->dens_sum + c->n, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(c->dens_cnt + c->n, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(c->dom_cnt + c->n, 0, sizeof(uint32_t) * n, s));
    CK(cudaStreamSynchronize(s));
    c->n += n;
    invalidate_render(c);
    return GS_OK;
}

__global__ void k_mask_u8(const uint32_t* __restrict__ keep, int n, uint8_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = keep[i] ? 1 : 0;
}

int gs_set_initializer(gs_ctx* c, gs_mlp* mlp) {
    if (!c) return GS_ERR_ARG;
    c->init_mlp = mlp;
    return GS_OK;
}

int gs_insert(gs_ctx* c, const gs_camera* cam, const float* image, const float* pts, int n, int* n_ins,
              uint8_t* inserted_dev, void* stream) {
    if (!c || !n_ins) return GS_ERR_ARG;
    *n_ins = 0;
    if (n < 0 || (n > 0 && (!pts || !image || !cam))) return fail(c, GS_ERR_ARG, "bad insertion arguments");
    if (n == 0) return GS_OK;
    if ((int64_t)c->n + n > c->cap) return fail(c, GS_ERR_CAPACITY, "insertion could exceed the capacity");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    Temp t;
    float *img = nullptr, *stage = nullptr, *feat = nullptr;
    uint32_t *keep = nullptr, *pos = nullptr;
    const size_t HW = (size_t)cam->width * cam->height;
    if (!t.get(&img, 3 * HW) || !t.get(&stage, kParamRows * (size_t)n) || !t.get(&keep, (size_t)n) ||
        !t.get(&pos, (size_t)n) || !t.get(&feat, 80 * (size_t)n))
        return fail(c, GS_ERR_OOM, "temporary buffers");
    if (c->cfg.insert_tau > 0.f) {
        // distance rule: no render, only the camera (pixel colours of the plain initialisation)
        CamBatch b;
        const int code = prepare_views(c, cam, 1, b);
        if (code != GS_OK) return code;
    } else {
        const int code = gs_render(c, cam, 1, img, nullptr, nullptr, stream);
        if (code != GS_OK) return code;
    }
    CK(launch_insert_test(c, c->hcam[0], pts, n, image, keep, stage, s));
    if (c->init_mlp) CK(mlp_initialise(c->init_mlp, c->hcam[0], image, pts, n, stage, feat, s));
    if (inserted_dev) {
        k_mask_u8<<<(n + 255) / 256, 256, 0, s>>>(keep, n, inserted_dev);
        CK(cudaGetLastError());
    }
    CK(scan_u32(c, keep, pos, (uint32_t)n, c->dcount + 5, s));
    CK(launch_append(c, stage, n, keep, pos, s));
    CK(cudaMemcpyAsync(c->hcount + 5, c->dcount + 5, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n_ins = (int)c->hcount[5];
    c->n += *n_ins;
    invalidate_render(c);
    return GS_OK;
}

int gs_count_dominant(gs_ctx* c, const gs_camera* cams, int n_views, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!cams || n_views < 1 || n_views > c->cfg.max_views) return fail(c, GS_ERR_ARG, "bad views");
    if (c->n == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    const size_t pix = (size_t)n_views * cams[0].width * cams[0].height;
    Temp t;
    float* img = nullptr;
    int32_t* am = nullptr;
    if (!t.get(&img, 3 * pix) || !t.get(&am, pix)) return fail(c, GS_ERR_OOM, "temporary buffers");
    const int code = gs_render(c, cams, n_views, img, nullptr, am, stream);
    if (code != GS_OK) return code;
    CK(launch_count_dominant(c, am, pix, s));
    CK(cudaStreamSynchronize(s));
    return GS_OK;
}

int gs_densify(gs_ctx* c, const float* normals, int* n_split_out, void* stream) {
    if (!c || !n_split_out) return GS_ERR_ARG;
    *n_split_out = 0;
    if (c->n == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    Temp t;
    uint32_t *flags = nullptr, *pos = nullptr;
    if (!t.get(&flags, (size_t)c->n) || !t.get(&pos, (size_t)c->n)) return fail(c, GS_ERR_OOM, "temporary buffers");
    CK(launch_split_flags(c, flags, s));
    CK(scan_u32(c, flags, pos, (uint32_t)c->n, c->dcount + 5, s));
    CK(cudaMemcpyAsync(c->hcount + 5, c->dcount + 5, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t n_split = c->hcount[5];
    if ((int64_t)c->n + n_split > c->cap) return fail(c, GS_ERR_CAPACITY, "splitting would exceed the capacity");
    if (n_split > 0) {
        float *P2 = nullptr, *M2 = nullptr, *V2 = nullptr;
        const size_t sz = kParamRows * (size_t)c->cap;
        if (dalloc(&P2, sz) != cudaSuccess) return fail(c, GS_ERR_OOM, "split buffers");
        if (dalloc(&M2, sz) != cudaSuccess) {
            cudaFree(P2);
            return fail(c, GS_ERR_OOM, "split buffers");
        }
        if (dalloc(&V2, sz) != cudaSuccess) {
            cudaFree(P2);
            cudaFree(M2);
            return fail(c, GS_ERR_OOM, "split buffers");
        }
        cudaError_t e = launch_split_scatter(c, flags, pos, n_split, normals, P2, M2, V2, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(P2);
            cudaFree(M2);
            cudaFree(V2);
            return fail(c, GS_ERR_CUDA, "split", e);
        }
        cudaFree(c->params);
        cudaFree(c->adam_m);
        cudaFree(c->adam_v);
        c->params = P2;
        c->adam_m = M2;
        c->adam_v = V2;
        c->n += (int)n_split;
    }
    CK(cudaMemsetAsync(c->dens_sum, 0, sizeof(float) * c->cap, s));
    CK(cudaMemsetAsync(c->dens_cnt, 0, sizeof(float) * c->cap, s));
    CK(cudaMemsetAsync(c->dom_cnt, 0, sizeof(uint32_t) * c->cap, s));
    CK(cudaStreamSynchronize(s));
    *n_split_out = (int)n_split;
    invalidate_render(c);
    return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint and resume of the map state (format in gs.h).

namespace {

struct CkptHeader {
    char magic[8];
    uint32_t version, rows, n, adam_steps_device;
    int32_t adam_steps_host;
    uint32_t reserved;
    double beta_powers[2];
    uint64_t payload_bytes, checksum;
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header layout");
constexpr char kCkptMagic[8] = {'G', 'S', 'M', 'A', 'P', 'C', 'K', '1'};
constexpr uint32_t kCkptVersion = 1;
constexpr uint64_t kCkptBytesPerGaussian = 4ull * (3 * kParamRows + 3);

// FNV-1a, 64-bit (Fowler, Noll, Vo)
uint64_t fnv1a64(const unsigned char* p, size_t n) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

// Reads and checks a whole checkpoint; on success `payload` holds its arrays.
// Returns nullptr or the reason it is not a valid checkpoint.
const char* read_checkpoint(const char* path, CkptHeader& h, std::vector<unsigned char>& payload) {
    FILE* f = fopen(path, "rb");
    if (!f) return "cannot open the checkpoint file";
    const char* why = nullptr;
    if (fread(&h, sizeof(h), 1, f) != 1) why = "checkpoint shorter than its header";
    else if (memcmp(h.magic, kCkptMagic, sizeof(kCkptMagic)) != 0) why = "not a checkpoint of this library";
    else if (h.version != kCkptVersion) why = "unsupported checkpoint version";
    else if (h.rows != (uint32_t)kParamRows) why = "checkpoint parameter rows differ";
    else if (h.payload_bytes != kCkptBytesPerGaussian * h.n) why = "checkpoint payload size does not match n";
    if (!why) {
        payload.resize((size_t)h.payload_bytes);
        if (h.payload_bytes && fread(payload.data(), 1, payload.size(), f) != payload.size())
            why = "checkpoint payload truncated";
        else if (fgetc(f) != EOF) why = "trailing bytes after the checkpoint payload";
        else if (fnv1a64(payload.data(), payload.size()) != h.checksum) why = "checkpoint checksum mismatch";
    }
    fclose(f);
    return why;
}

}  // namespace

int gs_checkpoint_info(const char* path, int* n, int* version) {
    if (!path) return GS_ERR_ARG;
    CkptHeader h;
    std::vector<unsigned char> payload;
    if (read_checkpoint(path, h, payload)) return GS_ERR_IO;
    if (n) *n = (int)h.n;
    if (version) *version = (int)h.version;
    return GS_OK;
}

int gs_save(gs_ctx* c, const char* path, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!path) return fail(c, GS_ERR_ARG, "path is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(s));
    const size_t n = (size_t)c->n;
    CkptHeader h = {};
    memcpy(h.magic, kCkptMagic, sizeof(kCkptMagic));
    h.version = kCkptVersion;
    h.rows = kParamRows;
    h.n = (uint32_t)n;
    h.adam_steps_host = c->adam_t;
    h.payload_bytes = kCkptBytesPerGaussian * n;
    std::vector<unsigned char> payload((size_t)h.payload_bytes);
    float* rows = reinterpret_cast<float*>(payload.data());
    const float* rows_src[3] = {c->params, c->adam_m, c->adam_v};
    for (int a = 0; a < 3; ++a)
        if (n)
            CK(cudaMemcpy2D(rows + (size_t)a * kParamRows * n, sizeof(float) * n, rows_src[a], sizeof(float) * c->cap,
                            sizeof(float) * n, kParamRows, cudaMemcpyDeviceToHost));
    float* tail = rows + (size_t)3 * kParamRows * n;
    if (n) {
        CK(cudaMemcpy(tail, c->dens_sum, sizeof(float) * n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tail + n, c->dens_cnt, sizeof(float) * n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tail + 2 * n, c->dom_cnt, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    }
    CK(cudaMemcpy(h.beta_powers, c->adam_pw, sizeof(double) * 2, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&h.adam_steps_device, c->dcount + 4, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    h.checksum = fnv1a64(payload.data(), payload.size());
    FILE* f = fopen(path, "wb");
    if (!f) return fail(c, GS_ERR_IO, "cannot create the checkpoint file");
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 &&
              (payload.empty() || fwrite(payload.data(), 1, payload.size(), f) == payload.size());
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(c, GS_ERR_IO, "writing the checkpoint file failed");
    return GS_OK;
}

int gs_load(gs_ctx* c, const char* path, void* stream) {
    if (!c) return GS_ERR_ARG;
    if (!path) return fail(c, GS_ERR_ARG, "path is NULL");
    CkptHeader h;
    std::vector<unsigned char> payload;
    if (const char* why = read_checkpoint(path, h, payload)) return fail(c, GS_ERR_IO, why);
    if (h.n > (uint32_t)c->cap) return fail(c, GS_ERR_CAPACITY, "the checkpoint holds more Gaussians than the capacity");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(s));
    const size_t n = h.n;
    const float* rows = reinterpret_cast<const float*>(payload.data());
    float* rows_dst[3] = {c->params, c->adam_m, c->adam_v};
    CK(cudaMemsetAsync(c->adam_m, 0, sizeof(float) * kParamRows * c->cap, s));
    CK(cudaMemsetAsync(c->adam_v, 0, sizeof(float) * kParamRows * c->cap, s));
    CK(cudaMemsetAsync(c->dens_sum, 0, sizeof(float) * c->cap, s));
    CK(cudaMemsetAsync(c->dens_cnt, 0, sizeof(float) * c->cap, s));
    CK(cudaMemsetAsync(c->dom_cnt, 0, sizeof(uint32_t) * c->cap, s));
    CK(cudaStreamSynchronize(s));
    for (int a = 0; a < 3; ++a)
        if (n)
            CK(cudaMemcpy2D(rows_dst[a], sizeof(float) * c->cap, rows + (size_t)a * kParamRows * n, sizeof(float) * n,
                            sizeof(float) * n, kParamRows, cudaMemcpyHostToDevice));
    const float* tail = rows + (size_t)3 * kParamRows * n;
    if (n) {
        CK(cudaMemcpy(c->dens_sum, tail, sizeof(float) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->dens_cnt, tail + n, sizeof(float) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->dom_cnt, tail + 2 * n, sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(c->adam_pw, h.beta_powers, sizeof(double) * 2, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->dcount + 4, &h.adam_steps_device, sizeof(uint32_t), cudaMemcpyHostToDevice));
    c->n = (int)n;
    c->adam_t = h.adam_steps_host;
    c->n_views = 0;
    c->loss_ready = c->backward_ready = false;
    drop_graph(c);
    return GS_OK;
}
