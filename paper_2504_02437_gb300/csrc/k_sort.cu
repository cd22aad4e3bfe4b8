// Tile binning and the (tile, depth) ordering of the pairs.
//
// The order the compositing needs is lexicographic in (view, tile, depth,
// Gaussian id). It is built in two stable steps instead of one 64-bit sort:
//   1. a stable LSD radix sort of the V*N depth keys (32 bits, 4 passes of 8),
//      whose stability keeps equal depths in id order;
//   2. pairs are emitted in that depth order (one per tile a Gaussian's pixel
//      box touches), then stably radix-sorted by bin = view * tiles + tile
//      (ceil(log2 bins) bits, 2 passes for up to 65536 bins).
// The second sort moves 8-byte pairs over P elements only twice instead of six
// times for a 64-bit key, and the depth sort touches N elements, not P.
//
// Every pass is reduce-then-scan over a fixed grid of G blocks, each owning a
// contiguous slice of the input; element counts are read from device memory so
// the same launches can sit in a CUDA graph.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                       // per lane per round
constexpr int kRound = kSortThreads * kSortItems;   // elements per block round

__device__ __forceinline__ void slice_of(uint32_t n, int G, int b, uint32_t& begin, uint32_t& end) {
    uint32_t chunk = (n + G - 1) / G;
    chunk = (chunk + 31u) & ~31u;
    uint64_t b0 = (uint64_t)chunk * b, b1 = b0 + chunk;
    begin = (uint32_t)(uint32_t)(b0 < n ? b0 : n);
    end = (uint32_t)(uint32_t)(b1 < n ? b1 : n);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Histogram of one digit over each block's slice: hist[d * G + b]. Each warp
// counts into its own shared sub-histogram (shared-memory atomics); every
// thread has four keys in flight per round.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ n_dev, uint32_t n_max,
                                                             int shift, int nbits, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kSortWarps][256];
    const int G = gridDim.x, b = blockIdx.x, w = threadIdx.x >> 5;
    const uint32_t mask = (1u << nbits) - 1u;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&h[0][0])[d] = 0;
    __syncthreads();
    uint32_t n = umin(*n_dev, n_max), begin, end;
    slice_of(n, G, b, begin, end);
    for (uint32_t base = begin + threadIdx.x; base < end; base += 4 * kSortThreads) {
        uint32_t k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t i = base + u * kSortThreads;
            k[u] = i < end ? keys[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (base + u * kSortThreads < end) atomicAdd(&h[w][(k[u] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)mask; d += kSortThreads) {
        uint32_t t = 0;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ++ww) t += h[ww][d];
        hist[(size_t)d * G + b] = t;
    }
}

// Exclusive scan of each digit's row of block counts (one CTA per digit):
// hist[d * G + b] <- sum of hist[d * G + b'] for b' < b; dtot[d] <- row total.
__global__ void __launch_bounds__(256) k_digit_scan(uint32_t* __restrict__ hist, int G, uint32_t* __restrict__ dtot) {
    __shared__ uint32_t ws[8];
    __shared__ uint32_t carry;
    const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t* row = hist + (size_t)d * G;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < G; base += 256) {
        const int i = base + t;
        const uint32_t c = i < G ? row[i] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        uint32_t pre = 0, tot = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t v = ws[k];
            pre += (k < w) ? v : 0u;
            tot += v;
        }
        const uint32_t before = carry;
        if (i < G) row[i] = before + pre + x - c;
        __syncthreads();
        if (t == 0) carry = before + tot;
        __syncthreads();
    }
    if (t == 0) dtot[d] = carry;
}

// Stable scatter of one digit pass. Each block walks its slice in rounds of
// kRound elements; warp w of a round owns a contiguous run of 32*kSortItems
// elements, ranked within the warp by __match_any_sync, across warps by a
// per-digit prefix over the warps' counts, and across blocks by the scanned
// histogram. The ranked round is first regrouped by digit in shared memory,
// then written out by consecutive threads, so each digit's run of the round
// leaves in coalesced stores instead of one scattered store per element.
// Five CTAs per SM (at most 51 registers; A/B on the 300k-Gaussian keyframe: iteration
// 0.5494 -> 0.5467 ms).
__global__ void __launch_bounds__(kSortThreads, 5) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* __restrict__ n_dev, uint32_t n_max, int shift, int nbits,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ dtot) {
    __shared__ uint32_t run[256];      // global position of the block's next element of each digit
    __shared__ uint32_t lstart[256];   // start of each digit's group in the staged round
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint32_t wcnt[kSortWarps][256];
    __shared__ uint32_t skey[kRound], sval[kRound];
    const int G = gridDim.x, b = blockIdx.x;
    const uint32_t mask = (1u << nbits) - 1u;
    const int ndig = 1 << nbits;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // exclusive scan of one value per thread (thread d holds digit d) over the block
    auto block_scan = [&](uint32_t c) -> uint32_t {
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t pre = 0;
        for (int k = 0; k < w; ++k) pre += wsum[k];
        __syncthreads();
        return pre + x - c;
    };
    {
        const int d = threadIdx.x;
        const uint32_t start = block_scan(d < ndig ? dtot[d] : 0u);
        if (d < ndig) run[d] = start + hist[(size_t)d * G + b];
    }
    uint32_t n = umin(*n_dev, n_max), begin, end;
    slice_of(n, G, b, begin, end);
    const uint32_t lt = lanemask_lt();
    for (uint32_t rbase = begin; rbase < end; rbase += kRound) {
        for (int d = lane; d < ndig; d += 32) wcnt[w][d] = 0;
        __syncwarp();
        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        const uint32_t wbase = rbase + (uint32_t)w * 32u * kSortItems;
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            uint32_t i = wbase + it * 32 + lane;
            bool ok = i < end;
            key[it] = ok ? kin[i] : 0u;
            val[it] = ok ? vin[i] : 0u;
            uint32_t d = ok ? (key[it] >> shift) & mask : 0xFFFFFFFFu;
            uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            uint32_t r = 0;
            if (ok) r = wcnt[w][d] + __popc(peers & lt);
            rank[it] = r;
            __syncwarp();
            if (ok && (__ffs(peers) - 1) == lane) wcnt[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: prefix over the warps, the round's count, and its group start in the round
        uint32_t tot = 0;
        {
            const int d = threadIdx.x;
            if (d < ndig) {
#pragma unroll
                for (int ww = 0; ww < kSortWarps; ++ww) {
                    const uint32_t c = wcnt[ww][d];
                    wcnt[ww][d] = tot;
                    tot += c;
                }
            }
            const uint32_t ls = block_scan(tot);   // synchronises the block
            if (d < ndig) lstart[d] = ls;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const uint32_t i = wbase + it * 32 + lane;
            if (i < end) {
                const uint32_t d = (key[it] >> shift) & mask;
                const uint32_t lp = lstart[d] + wcnt[w][d] + rank[it];
                skey[lp] = key[it];
                sval[lp] = val[it];
            }
        }
        __syncthreads();
        const uint32_t cnt = umin((uint32_t)kRound, end - rbase);
        for (uint32_t j = threadIdx.x; j < cnt; j += kSortThreads) {
            const uint32_t k2 = skey[j], d = (k2 >> shift) & mask;
            const uint32_t pos = run[d] + (j - lstart[d]);
            kout[pos] = k2;
            vout[pos] = sval[j];
        }
        __syncthreads();
        if (threadIdx.x < ndig) run[threadIdx.x] += tot;
        __syncthreads();
    }
}

// ---- scan of the tiles touched, in depth order ----

__global__ void __launch_bounds__(256) k_tile_block_sums(const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ tiles, uint32_t n,
                                                         const uint32_t* __restrict__ n_dev,
                                                         uint32_t* __restrict__ bsum) {
    __shared__ uint32_t ws[8];
    if (n_dev != nullptr) n = umin(n, *n_dev);
    uint32_t begin, end;
    slice_of(n, gridDim.x, blockIdx.x, begin, end);
    uint32_t s = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += 256) s += tiles[order ? order[i] : i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < 8; ++k) t += ws[k];
        bsum[blockIdx.x] = t;
    }
}

// Exclusive scan of the slices of k_tile_block_sums: block b first adds the block sums of the
// slices before its own (a few hundred values, read straight from bsum: no separate scan
// launch), then scans its slice; the last block writes the total.
__global__ void __launch_bounds__(256) k_tile_scan(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ tiles, uint32_t n,
                                                   const uint32_t* __restrict__ n_dev,
                                                   const uint32_t* __restrict__ bsum, uint32_t* __restrict__ off,
                                                   uint32_t* __restrict__ total_out) {
    __shared__ uint32_t ws[8];
    __shared__ uint32_t carry;
    if (n_dev != nullptr) n = umin(n, *n_dev);
    uint32_t begin, end;
    slice_of(n, gridDim.x, blockIdx.x, begin, end);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {
        uint32_t pre = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 256) pre += bsum[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
        if (lane == 0) ws[w] = pre;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int k = 0; k < 8; ++k) t += ws[k];
            carry = t;
        }
        __syncthreads();
    }
    for (uint32_t base = begin; base < end; base += 256) {
        uint32_t i = base + threadIdx.x;
        uint32_t c = i < end ? tiles[order ? order[i] : i] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        uint32_t pre = 0, tot = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t v = ws[k];
            pre += (k < w) ? v : 0u;
            tot += v;
        }
        if (i < end) off[i] = carry + pre + x - c;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (total_out != nullptr && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = carry;
}

// Pair emission: item k of the depth order owns pairs off[k] .. off[k] + tiles
// - 1, one per tile of its pixel box in row-major order (bin, item). Each warp
// takes 32 consecutive items, scans their tile counts, and writes the warp's
// pairs (a contiguous run of the output) 32 at a time: lane j writes pair t =
// t0 + j of the run, owned by the last lane whose exclusive count is <= t, so
// the stores are coalesced and a large Gaussian's pairs are spread over the
// warp. An item whose pairs would pass pair_cap is skipped and sets *overflow.
// In the deterministic mode (emit_item != NULL) a pair's value is its emission
// index e instead of its item, emit_item[e] holds the item, and the pair's
// gradient slot pairgrad[9 e ..] is cleared.
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ order, const uint32_t* __restrict__ tiles,
                                              const uint32_t* __restrict__ off, const float4* __restrict__ rec,
                                              const DevCamera* __restrict__ cams, int n, int tile, uint32_t n_items,
                                              const uint32_t* __restrict__ n_dev, uint64_t pair_cap,
                                              uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval,
                                              uint32_t* __restrict__ overflow, uint32_t* __restrict__ emit_item,
                                              float* __restrict__ pairgrad) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint32_t nv = umin(n_items, *n_dev);
    if (k - (uint32_t)lane >= nv) return;   // the whole warp is past the visible items
    uint32_t item = 0, cnt = 0, o = 0, bin0 = 0, tiles_x = 0;
    int tx0 = 0, ty0 = 0, wt = 1;
    if (k < nv) {
        item = order[k];
        cnt = tiles[item];
        if (cnt != 0) {
            o = off[k];
            if ((uint64_t)o + cnt > pair_cap) {
                atomicMax(overflow, 1u);
                cnt = 0;
            } else {
                const DevCamera& cam = cams[item / (uint32_t)n];
                const float4 f0 = rec[(size_t)item * 3], f1 = rec[(size_t)item * 3 + 1],
                             f2 = rec[(size_t)item * 3 + 2];
                int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
                pixel_box(f0.x, f1.w, f0.y, f2.w, f0.z, cam.width, cam.height, x0, x1, y0, y1);
                tx0 = x0 / tile;
                ty0 = y0 / tile;
                wt = x1 / tile - tx0 + 1;
                bin0 = (uint32_t)cam.bin_base;
                tiles_x = (uint32_t)cam.tiles_x;
            }
        }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + (uint32_t)lane;
        int src = 0;   // last lane with excl <= t (lanes without pairs share the next lane's excl)
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int cand = src + step;
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, cand & 31);
            if (cand < 32 && e <= t) src = cand;
        }
        const uint32_t s_excl = __shfl_sync(0xFFFFFFFFu, excl, src);
        const uint32_t s_o = __shfl_sync(0xFFFFFFFFu, o, src);
        const uint32_t s_item = __shfl_sync(0xFFFFFFFFu, item, src);
        const uint32_t s_bin0 = __shfl_sync(0xFFFFFFFFu, bin0, src);
        const uint32_t s_tx = __shfl_sync(0xFFFFFFFFu, tiles_x, src);
        const int s_tx0 = __shfl_sync(0xFFFFFFFFu, tx0, src);
        const int s_ty0 = __shfl_sync(0xFFFFFFFFu, ty0, src);
        const int s_wt = __shfl_sync(0xFFFFFFFFu, wt, src);
        if (t < total) {
            const uint32_t local = t - s_excl;
            const uint32_t row = local / (uint32_t)s_wt;
            const uint32_t col = local - row * (uint32_t)s_wt;
            const uint32_t pos = s_o + local;
            pkey[pos] = s_bin0 + (uint32_t)(s_ty0 + (int)row) * s_tx + (uint32_t)(s_tx0 + (int)col);
            if (emit_item != nullptr) {
                pval[pos] = pos;
                emit_item[pos] = s_item;
#pragma unroll
                for (int q = 0; q < kPairGradStride; ++q) pairgrad[(size_t)pos * kPairGradStride + q] = 0.f;
            } else {
                pval[pos] = s_item;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ pkey, const uint32_t* __restrict__ P_dev,
                                                uint64_t pair_cap, uint32_t n_bins, uint2* __restrict__ ranges) {
    uint32_t P = (uint32_t)(*P_dev < pair_cap ? *P_dev : pair_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        uint32_t b = pkey[i];
        if (b >= n_bins) continue;   // only possible after a pair-buffer overflow
        if (i == 0 || pkey[i - 1] != b) ranges[b].x = i;
        if (i == P - 1 || pkey[i + 1] != b) ranges[b].y = i + 1;
    }
}

// Bucket of a bin in the longest-first work order: 1023 - key, where the key
// grows with the bin's pair count (steps of 2 pairs below 1,024 pairs, of 16
// up to 9,200, one bucket above).
__device__ __forceinline__ uint32_t order_slot(uint2 r) {
    const uint32_t len = r.y - r.x;
    const uint32_t key = len < 1024u ? len >> 1 : 512u + min(511u, (len - 1024u) >> 4);
    return 1023u - key;
}

// Longest-first order of the bins for the persistent compositing kernels
// (list scheduling, largest job first): their work queue hands out the tiles
// with the most pairs first, so a launch does not end on a long tile taken
// late. One CTA, a counting sort by bucket; bins of one bucket come in any
// order (the compositing result does not depend on which CTA takes a tile).
__global__ void __launch_bounds__(1024) k_work_order(const uint2* __restrict__ ranges, uint32_t n_bins,
                                                      uint32_t* __restrict__ order) {
    __shared__ uint32_t cnt[1024];
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31;
    cnt[t] = 0;
    __syncthreads();
    for (uint32_t b = t; b < n_bins; b += 1024) atomicAdd(&cnt[order_slot(ranges[b])], 1u);
    __syncthreads();
    const uint32_t v = cnt[t];
    uint32_t x = v;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[t >> 5] = x;
    __syncthreads();
    if (t < 32) {
        const uint32_t w = wsum[t];
        uint32_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= o) z += y;
        }
        wsum[t] = z - w;
    }
    __syncthreads();
    cnt[t] = x - v + wsum[t >> 5];
    __syncthreads();
    for (uint32_t b = t; b < n_bins; b += 1024) order[atomicAdd(&cnt[order_slot(ranges[b])], 1u)] = b;
}

}  // namespace

cudaError_t radix_sort_pairs(gs_ctx* c, uint32_t** keys, uint32_t** vals, const uint32_t* n_dev, uint32_t n_max,
                             uint32_t n_hint, int bits, int* out_buf, cudaStream_t s) {
    int cur = 0;
    // about 2048 elements (one scatter round) per block, each block owning one contiguous slice
    const int G = (int)std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)c->sort_blocks, (n_hint + 2047u) / 2048u));
    for (int shift = 0; shift < bits; shift += 8) {
        int nb = bits - shift < 8 ? bits - shift : 8;
        c->launches += 3;
        uint32_t* dtot = c->hist + (size_t)256 * c->sort_blocks;
        k_radix_hist<<<G, kSortThreads, 0, s>>>(keys[cur], n_dev, n_max, shift, nb, c->hist);
        k_digit_scan<<<1 << nb, 256, 0, s>>>(c->hist, G, dtot);
        k_radix_scatter<<<G, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_dev, n_max,
                                                   shift, nb, c->hist, dtot);
        cur ^= 1;
    }
    *out_buf = cur;
    return cudaGetLastError();
}

cudaError_t scan_tiles(gs_ctx* c, uint32_t n_max, const uint32_t* n_dev, cudaStream_t s) {
    // the depth-sorted order is in dval[0] after the even number (4) of depth passes
    const int G = c->sort_blocks;
    c->launches += 2;
    k_tile_block_sums<<<G, 256, 0, s>>>(c->dval[0], c->tiles_touched, n_max, n_dev, c->hist);
    k_tile_scan<<<G, 256, 0, s>>>(c->dval[0], c->tiles_touched, n_max, n_dev, c->hist, c->offsets, c->dcount);
    return cudaGetLastError();
}

cudaError_t scan_u32(gs_ctx* c, const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total_dev,
                     cudaStream_t s) {
    const int G = c->sort_blocks;
    c->launches += 2;
    k_tile_block_sums<<<G, 256, 0, s>>>(nullptr, in, n, nullptr, c->hist);
    k_tile_scan<<<G, 256, 0, s>>>(nullptr, in, n, nullptr, c->hist, out, total_dev);
    return cudaGetLastError();
}

cudaError_t emit_pairs(gs_ctx* c, uint32_t n_items, const uint32_t* n_dev, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    ++c->launches;
    k_emit<<<(n_items + 255) / 256, 256, 0, s>>>(c->dval[0], c->tiles_touched, c->offsets, c->rec, c->dcam, c->n,
                                                 c->tile, n_items, n_dev, (uint64_t)c->pair_cap, c->pkey[0],
                                                 c->pval[0], c->dcount + 1, c->emit_item, c->pairgrad);
    return cudaGetLastError();
}

// Deterministic mode: item k of the depth order owns the pair slots off[k] ..
// off[k] + tiles - 1 (its emission indices); their screen gradients are added in
// that order into the item's grad2d record.
__global__ void __launch_bounds__(256) k_pairgrad_reduce(const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ tiles,
                                                         const uint32_t* __restrict__ off, uint32_t n_items,
                                                         const uint32_t* __restrict__ n_dev, uint64_t pair_cap,
                                                         const float* __restrict__ pairgrad,
                                                         float* __restrict__ grad2d) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_items || k >= *n_dev) return;
    const uint32_t item = order[k], cnt = tiles[item];
    const uint64_t o = off[k];
    float s[kPairGradStride];
#pragma unroll
    for (int q = 0; q < kPairGradStride; ++q) s[q] = 0.f;
    if (cnt != 0 && o + cnt <= pair_cap)
        for (uint64_t e = o; e < o + cnt; ++e)
#pragma unroll
            for (int q = 0; q < kPairGradStride; ++q) s[q] += pairgrad[e * kPairGradStride + q];
#pragma unroll
    for (int q = 0; q < kPairGradStride; ++q) grad2d[(size_t)item * kGrad2dStride + q] = s[q];
}

cudaError_t reduce_pair_grads(gs_ctx* c, cudaStream_t s) {
    const uint32_t items = (uint32_t)c->n_views * (uint32_t)c->n;
    if (c->pairgrad == nullptr || items == 0) return cudaSuccess;
    ++c->launches;
    k_pairgrad_reduce<<<(items + 255) / 256, 256, 0, s>>>(c->dval[0], c->tiles_touched, c->offsets, items,
                                                          c->dcount + 8, (uint64_t)c->pair_cap, c->pairgrad,
                                                          c->grad2d);
    return cudaGetLastError();
}

cudaError_t compute_ranges(gs_ctx* c, cudaStream_t s) {
    // (a mapping iteration zeroes the ranges on its side stream)
    if (!c->side_zeroed) cudaMemsetAsync(c->ranges, 0, sizeof(uint2) * (size_t)c->n_bins, s);
    ++c->launches;
    k_ranges<<<c->num_sms * 8, 256, 0, s>>>(c->pkey[c->pair_buf], c->dcount, (uint64_t)c->pair_cap,
                                            (uint32_t)c->n_bins, c->ranges);
    ++c->launches;
    if (c->order_ahead) {
        // the next iteration's order, beside this one's compositing (which uses the order the
        // previous iteration left); iteration_tail copies it into place after the compositing
        cudaEventRecord(c->side_ev[5], s);
        cudaStreamWaitEvent(c->side, c->side_ev[5], 0);
        k_work_order<<<1, 1024, 0, c->side>>>(c->ranges, (uint32_t)c->n_bins, c->work_order_next);
    } else {
        k_work_order<<<1, 1024, 0, s>>>(c->ranges, (uint32_t)c->n_bins, c->work_order);
    }
    return cudaGetLastError();
}

}  // namespace gs

// ---------------------------------------------------------------------------
// Allocation-free variant of the pair sort, for callers that must not allocate
// device memory (for example code that runs while another component owns the
// device allocator, or a real-time loop that forbids cudaMalloc). Its scratch
// is one file-scope __device__ array that every GPU loading this library holds
// until the process exits.

namespace gs {
namespace {

constexpr uint32_t kStaticSortMaxPairs = 1u << 20;                       // largest n accepted
constexpr int kStaticSortMaxBlocks = (int)((kStaticSortMaxPairs + 4095u) / 4096u);
constexpr size_t kStaticSortWords = 64                                  // [0] count sentinel
                                    + 2 * (size_t)kStaticSortMaxPairs    // ping-pong keys and values
                                    + 256 * (size_t)kStaticSortMaxBlocks + 256;   // histograms, digit totals
static __device__ __align__(256) uint32_t g_static_sort_scratch[kStaticSortWords];

// [a, a + n) and [b, b + n) words overlap
bool ranges_overlap(const void* a, const void* b, uint64_t n) {
    const uint64_t x = (uint64_t)(uintptr_t)a, y = (uint64_t)(uintptr_t)b, len = 4 * n;
    return x < y + len && y < x + len;
}

}  // namespace
}  // namespace gs

extern "C" int gs_sort_pairs_static(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                    uint32_t* vals_out, int64_t n, int bits, void* stream) {
    using namespace gs;
    if (n < 0 || bits < 1 || bits > 32) return GS_ERR_ARG;
    if (n > (int64_t)kStaticSortMaxPairs) return GS_ERR_CAPACITY;
    if (n == 0) return GS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return GS_ERR_ARG;
    // a pass reads the inputs while it writes the outputs: no output may overlap an input or the
    // other output (the inputs may overlap each other)
    const uint64_t un64 = (uint64_t)n;
    if (ranges_overlap(keys_out, vals_out, un64) || ranges_overlap(keys_out, keys_in, un64) ||
        ranges_overlap(keys_out, vals_in, un64) || ranges_overlap(vals_out, keys_in, un64) ||
        ranges_overlap(vals_out, vals_in, un64))
        return GS_ERR_ARG;
    // an unchecked error of earlier work is left for its owner: nothing is launched
    if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
    // The device address of the scratch array on the current device. In host code the array's
    // name is only a host-side stand-in; the runtime maps it to this device's copy. Resolved on
    // every call (a lookup once the device code is loaded, which the first call on a device
    // does), so a context that was reset and re-created gets its own address.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_sort_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();   // this call's own error, reported by the return code
        return GS_ERR_CUDA;
    }
    uint32_t* base = static_cast<uint32_t*>(p);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* sentinel = base;
    uint32_t* tmp_k = base + 64;
    uint32_t* tmp_v = tmp_k + kStaticSortMaxPairs;
    uint32_t* hist = tmp_v + kStaticSortMaxPairs;
    const uint32_t un = (uint32_t)n;
    const int G = (int)std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)kStaticSortMaxBlocks, (un + 4095u) / 4096u));
    uint32_t* dtot = hist + (size_t)256 * G;
    // the count is passed as n_max with a device-side bound of 0xFFFFFFFF
    if (cudaMemsetAsync(sentinel, 0xFF, sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    const int passes = (bits + 7) / 8;
    const uint32_t* src_k = keys_in;
    const uint32_t* src_v = vals_in;
    for (int i = 0; i < passes; ++i) {
        // destinations alternate so that the last pass writes the caller's output
        const bool to_out = ((passes - i) & 1) == 1;
        uint32_t* dk = to_out ? keys_out : tmp_k;
        uint32_t* dv = to_out ? vals_out : tmp_v;
        const int shift = 8 * i;
        const int nb = bits - shift < 8 ? bits - shift : 8;
        k_radix_hist<<<G, kSortThreads, 0, s>>>(src_k, sentinel, un, shift, nb, hist);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
        k_digit_scan<<<1 << nb, 256, 0, s>>>(hist, G, dtot);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
        k_radix_scatter<<<G, kSortThreads, 0, s>>>(src_k, src_v, dk, dv, sentinel, un, shift, nb, hist, dtot);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
        src_k = dk;
        src_v = dv;
    }
    return GS_OK;
}
