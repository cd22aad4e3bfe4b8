// Map management: initialisation from back-projected points (Eq. 6), dynamic
// insertion gated by rendered opacity (Eq. 7 reading) and densification by
// splitting (Section 3.2). These run once per keyframe, not per iteration.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

// 3 smallest squared distances from q to the reference points (one CTA per query).
// ref is planar [3][ref_stride]; skip index `self` (or -1). Returns the RMS of
// those distances (0.01 if there is no reference point) to every thread, and
// the smallest squared distance (+inf if none) in *dmin2 of thread 0.
__device__ float knn3_rms(const float* __restrict__ ref, int ref_stride, int n_ref, float qx, float qy, float qz,
                          int self, float* dmin2) {
    __shared__ float best[256 * 3];
    float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY;
    for (int j = threadIdx.x; j < n_ref; j += blockDim.x) {
        if (j == self) continue;
        float dx = ref[j] - qx, dy = ref[ref_stride + j] - qy, dz = ref[2 * ref_stride + j] - qz;
        float d = dx * dx + dy * dy + dz * dz;
        if (d < b2) {
            if (d < b1) {
                b2 = b1;
                if (d < b0) {
                    b1 = b0;
                    b0 = d;
                } else {
                    b1 = d;
                }
            } else {
                b2 = d;
            }
        }
    }
    best[threadIdx.x * 3 + 0] = b0;
    best[threadIdx.x * 3 + 1] = b1;
    best[threadIdx.x * 3 + 2] = b2;
    __syncthreads();
    __shared__ float rms;
    if (threadIdx.x == 0) {
        float c0 = INFINITY, c1 = INFINITY, c2 = INFINITY;
        for (int k = 0; k < (int)blockDim.x * 3; ++k) {
            float d = best[k];
            if (d < c2) {
                if (d < c1) {
                    c2 = c1;
                    if (d < c0) {
                        c1 = c0;
                        c0 = d;
                    } else {
                        c1 = d;
                    }
                } else {
                    c2 = d;
                }
            }
        }
        *dmin2 = c0;
        int cnt = (c0 < INFINITY) + (c1 < INFINITY) + (c2 < INFINITY);
        float s = (cnt > 0 ? c0 : 0.f) + (cnt > 1 ? c1 : 0.f) + (cnt > 2 ? c2 : 0.f);
        rms = cnt > 0 ? sqrtf(s / (float)cnt) : 0.01f;
    }
    __syncthreads();
    return rms;
}

// Plain initialisation of one new Gaussian per block.
__global__ void __launch_bounds__(256) k_init_points(const float* __restrict__ pts, const float* __restrict__ rgb,
                                                     const float* __restrict__ ref, int ref_stride, int n_ref,
                                                     int ref_is_self, float* __restrict__ out, int out_stride) {
    int i = blockIdx.x;
    float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    float dmin2;
    float rms = knn3_rms(ref, ref_stride, n_ref, x, y, z, ref_is_self ? i : -1, &dmin2);
    if (threadIdx.x == 0) {
        float ls = fminf(fmaxf(logf(fmaxf(rms, 1e-30f)), -7.f), -1.f);
        const float v[kParamRows] = {x, y, z, ls, ls, ls, 1.f, 0.f, 0.f, 0.f, 0.f, rgb[3 * i], rgb[3 * i + 1],
                                     rgb[3 * i + 2]};
        for (int r = 0; r < kParamRows; ++r) out[(size_t)r * out_stride + i] = v[r];
    }
}

// Insertion test of point i. Opacity gate (tau2 = 0): keep[i] = 0 iff the point
// projects, in front of the camera, to a pixel whose rendered opacity 1 - T
// exceeds the threshold. Distance rule (tau2 = tau^2 > 0, Eq. 7 as its text
// states it): keep[i] = 1 iff the nearest existing mean is farther than tau
// (T is not read). Also stages the plain initial parameters [14][n].
__global__ void __launch_bounds__(256) k_insert_test(DevCamera cam, float near_z, float thresh, float tau2,
                                                     const float* __restrict__ pts, const float* __restrict__ T,
                                                     const float* __restrict__ image, const float* __restrict__ ref,
                                                     int ref_stride, int n_ref, uint32_t* __restrict__ keep,
                                                     float* __restrict__ stage, int n) {
    int i = blockIdx.x;
    float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    float dmin2 = INFINITY;
    float rms = knn3_rms(ref, ref_stride, n_ref, x, y, z, -1, &dmin2);
    if (threadIdx.x != 0) return;
    float tx = cam.R[0] * x + cam.R[1] * y + cam.R[2] * z + cam.t[0];
    float ty = cam.R[3] * x + cam.R[4] * y + cam.R[5] * z + cam.t[1];
    float tz = cam.R[6] * x + cam.R[7] * y + cam.R[8] * z + cam.t[2];
    bool front = tz > near_z;
    float zz = front ? tz : 1.f;
    float u = cam.fx * tx / zz + cam.cx, v = cam.fy * ty / zz + cam.cy;
    float pxf = floorf(u + 0.5f), pyf = floorf(v + 0.5f);
    bool inside = front && pxf >= 0.f && pxf < (float)cam.width && pyf >= 0.f && pyf < (float)cam.height;
    int px = inside ? (int)pxf : 0, py = inside ? (int)pyf : 0;
    size_t HW = (size_t)cam.width * cam.height, pix = (size_t)py * cam.width + px;
    bool skip = tau2 > 0.f ? !(dmin2 > tau2) : (inside && (1.f - T[pix]) > thresh);
    keep[i] = skip ? 0u : 1u;
    float ls = fminf(fmaxf(logf(fmaxf(rms, 1e-30f)), -7.f), -1.f);
    const float vals[kParamRows] = {x, y, z, ls, ls, ls, 1.f, 0.f, 0.f, 0.f, 0.f,
                                    image[pix], image[HW + pix], image[2 * HW + pix]};
    for (int r = 0; r < kParamRows; ++r) stage[(size_t)r * n + i] = vals[r];
}

__global__ void __launch_bounds__(256) k_append(const float* __restrict__ stage, int n_stage,
                                                const uint32_t* __restrict__ keep, const uint32_t* __restrict__ pos,
                                                float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                                                float* __restrict__ dsum, float* __restrict__ dcnt,
                                                uint32_t* __restrict__ dom, int base, int cap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_stage || !keep[i]) return;
    int d = base + (int)pos[i];
    for (int r = 0; r < kParamRows; ++r) {
        P[(size_t)r * cap + d] = stage[(size_t)r * n_stage + i];
        M[(size_t)r * cap + d] = 0.f;
        V[(size_t)r * cap + d] = 0.f;
    }
    dsum[d] = 0.f;
    dcnt[d] = 0.f;
    dom[d] = 0u;
}

// Split mask: the gradient criterion, or (sigma > 0) more than sigma dominated
// pixels (Eq. 9 split mask M).
__global__ void __launch_bounds__(256) k_split_flags(const float* __restrict__ dsum, const float* __restrict__ dcnt,
                                                     const uint32_t* __restrict__ dom, int n, float thresh,
                                                     float sigma, uint32_t* __restrict__ flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c = dcnt[i];
    float mean = c > 0.f ? dsum[i] / c : 0.f;
    const bool clear = sigma > 0.f && (float)dom[i] > sigma;
    flags[i] = (mean > thresh || clear) ? 1u : 0u;
}

// Eq. 8-9: every pixel whose largest blend weight belongs to Gaussian a adds one
// to a's dominated-pixel count (argmax -1: no Gaussian).
__global__ void __launch_bounds__(256) k_count_dominant(const int32_t* __restrict__ argmax, size_t n_pix, int n,
                                                        uint32_t* __restrict__ dom) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_pix; i += (size_t)gridDim.x * blockDim.x) {
        const int a = argmax[i];
        if (a >= 0 && a < n) atomicAdd(dom + a, 1u);
    }
}

// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// standard normal by the Box-Muller transform of two counter-based uniforms
__device__ float normal_at(uint64_t seed, uint64_t counter) {
    uint64_t a = splitmix64(seed ^ (2 * counter)), b = splitmix64(seed ^ (2 * counter + 1));
    float u1 = ((float)(a >> 40) + 0.5f) * (1.0f / 16777216.0f);
    float u2 = (float)(b >> 40) * (1.0f / 16777216.0f);
    return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// Survivors move to pos_s = i - (split parents before i); children of the
// k-th split parent go to n_surv + 2k and n_surv + 2k + 1.
__global__ void __launch_bounds__(256) k_split_scatter(const float* __restrict__ P, const float* __restrict__ M,
                                                       const float* __restrict__ V, int n, int cap,
                                                       const uint32_t* __restrict__ flags,
                                                       const uint32_t* __restrict__ pos, uint32_t n_split,
                                                       const float* __restrict__ normals, uint64_t seed,
                                                       float log_factor, float* __restrict__ P2,
                                                       float* __restrict__ M2, float* __restrict__ V2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t before = pos[i];
    float p[kParamRows];
    for (int r = 0; r < kParamRows; ++r) p[r] = P[(size_t)r * cap + i];
    if (!flags[i]) {
        int d = i - (int)before;
        for (int r = 0; r < kParamRows; ++r) {
            P2[(size_t)r * cap + d] = p[r];
            M2[(size_t)r * cap + d] = M[(size_t)r * cap + i];
            V2[(size_t)r * cap + d] = V[(size_t)r * cap + i];
        }
        return;
    }
    int n_surv = n - (int)n_split;
    float qq = sqrtf(p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]);
    float w = p[6] / qq, x = p[7] / qq, y = p[8] / qq, z = p[9] / qq;
    float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                  2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                  2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float s[3] = {expf(p[3]), expf(p[4]), expf(p[5])};
    for (int k = 0; k < 2; ++k) {
        float zn[3];
        for (int a = 0; a < 3; ++a)
            zn[a] = normals ? normals[(size_t)i * 6 + k * 3 + a] : normal_at(seed, (uint64_t)i * 6 + k * 3 + a);
        int d = n_surv + 2 * (int)before + k;
        for (int r = 0; r < kParamRows; ++r) {
            float v = p[r];
            if (r < 3) v = p[r] + R[r * 3 + 0] * s[0] * zn[0] + R[r * 3 + 1] * s[1] * zn[1] + R[r * 3 + 2] * s[2] * zn[2];
            else if (r < 6) v = p[r] - log_factor;
            P2[(size_t)r * cap + d] = v;
            M2[(size_t)r * cap + d] = 0.f;
            V2[(size_t)r * cap + d] = 0.f;
        }
    }
}

}  // namespace

cudaError_t launch_init_points(gs_ctx* c, const float* pts, const float* rgb, int n, const float* ref, int ref_stride,
                               int n_ref, int ref_is_self, float* out_params, int out_stride, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    ++c->launches;
    k_init_points<<<n, 256, 0, s>>>(pts, rgb, ref, ref_stride, n_ref, ref_is_self, out_params, out_stride);
    return cudaGetLastError();
}

namespace {
__global__ void k_points_planar(const float* __restrict__ pts, int n, float* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = pts[3 * i];
    out[n + i] = pts[3 * i + 1];
    out[2 * n + i] = pts[3 * i + 2];
}
}  // namespace

cudaError_t launch_points_planar(const float* pts, int n, float* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_points_planar<<<(n + 255) / 256, 256, 0, s>>>(pts, n, out);
    return cudaGetLastError();
}

cudaError_t launch_insert_test(gs_ctx* c, const DevCamera& cam, const float* pts, int n, const float* image,
                               uint32_t* keep, float* stage, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    ++c->launches;
    const float tau2 = c->cfg.insert_tau > 0.f ? c->cfg.insert_tau * c->cfg.insert_tau : 0.f;
    k_insert_test<<<n, 256, 0, s>>>(cam, c->cfg.near_z, c->cfg.insert_opacity, tau2, pts, c->T_final, image,
                                    c->params, c->cap, c->n, keep, stage, n);
    return cudaGetLastError();
}

cudaError_t launch_append(gs_ctx* c, const float* stage, int n_stage, const uint32_t* keep, const uint32_t* pos,
                          cudaStream_t s) {
    if (n_stage == 0) return cudaSuccess;
    ++c->launches;
    k_append<<<(n_stage + 255) / 256, 256, 0, s>>>(stage, n_stage, keep, pos, c->params, c->adam_m, c->adam_v,
                                                   c->dens_sum, c->dens_cnt, c->dom_cnt, c->n, c->cap);
    return cudaGetLastError();
}

cudaError_t launch_split_flags(gs_ctx* c, uint32_t* flags, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    ++c->launches;
    k_split_flags<<<(c->n + 255) / 256, 256, 0, s>>>(c->dens_sum, c->dens_cnt, c->dom_cnt, c->n,
                                                     c->cfg.split_thresh, c->cfg.clarity_sigma, flags);
    return cudaGetLastError();
}

cudaError_t launch_count_dominant(gs_ctx* c, const int32_t* argmax, size_t n_pix, cudaStream_t s) {
    if (n_pix == 0 || c->n == 0) return cudaSuccess;
    ++c->launches;
    const int grid = (int)std::min<size_t>((n_pix + 255) / 256, (size_t)c->num_sms * 8);
    k_count_dominant<<<grid, 256, 0, s>>>(argmax, n_pix, c->n, c->dom_cnt);
    return cudaGetLastError();
}

cudaError_t launch_split_scatter(gs_ctx* c, const uint32_t* flags, const uint32_t* pos, uint32_t n_split,
                                 const float* normals, float* P2, float* M2, float* V2, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    ++c->launches;
    k_split_scatter<<<(c->n + 255) / 256, 256, 0, s>>>(c->params, c->adam_m, c->adam_v, c->n, c->cap, flags, pos,
                                                       n_split, normals, c->cfg.seed, logf(c->cfg.split_factor), P2,
                                                       M2, V2);
    return cudaGetLastError();
}

}  // namespace gs
