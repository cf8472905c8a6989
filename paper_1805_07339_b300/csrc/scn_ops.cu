// Sequence operations around the per-frame kernels: spacing (the inverse of a
// sampling op), slicing at boundaries and a stencil that respects slices, and
// the per-shot montage.
//
// Paper anchors: sampling/spacing operations insert "fill" elements to align
// sequences sampled at different rates (Sec. 3.2); slicing partitions a
// sequence so that stencils do not reach across boundaries, e.g. shots
// (Sec. 3.2); film summaries show one frame per detected shot (Sec. 5.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "scn_internal.h"

namespace scn {
namespace {

// Spacing workspace of a sequence: its distinct sampled frames in ascending
// order and, for each, the sequence element that supplies it (the last one
// when a frame is sampled more than once).
struct SpaceWs {
    void* block = nullptr;
    int32_t* frame = nullptr;  // [m]
    int32_t* elem = nullptr;   // [m]
    uint8_t* fill = nullptr;   // [kMaxElem]
    int64_t m = 0;
};

constexpr int kMaxElem = 1024;

scn_status ensure_space_ws(scn_seq* s, SpaceWs*& ws) {
    ws = static_cast<SpaceWs*>(s->space_ws);
    if (ws) return SCN_OK;
    std::vector<std::pair<int64_t, int64_t>> fk(s->n);
    for (int64_t k = 0; k < s->n; ++k) fk[k] = {s->frames[k], k};
    std::sort(fk.begin(), fk.end());  // by frame, then element: the last of a run is the largest k
    std::vector<int32_t> f, e;
    for (size_t i = 0; i < fk.size(); ++i) {
        if (i + 1 < fk.size() && fk[i + 1].first == fk[i].first) continue;
        f.push_back(static_cast<int32_t>(fk[i].first));
        e.push_back(static_cast<int32_t>(fk[i].second));
    }
    ws = new (std::nothrow) SpaceWs;
    if (!ws) return SCN_ENOMEM;
    const size_t m = f.size(), up = ((std::max<size_t>(m, 1) * 4) + 255) & ~size_t(255);
    cudaError_t err = obj_alloc(&ws->block, 2 * up + kMaxElem);
    if (err == cudaSuccess && m) err = obj_upload(ws->block, f.data(), m * 4);
    if (err == cudaSuccess && m) err = obj_upload(static_cast<char*>(ws->block) + up, e.data(), m * 4);
    if (err == cudaSuccess) err = obj_finish();  // f and e are host vectors of this call
    if (err != cudaSuccess) {
        set_cuda_error(err);
        obj_free(ws->block);
        delete ws;
        ws = nullptr;
        return SCN_ECUDA;
    }
    ws->frame = static_cast<int32_t*>(ws->block);
    ws->elem = reinterpret_cast<int32_t*>(static_cast<char*>(ws->block) + up);
    ws->fill = reinterpret_cast<uint8_t*>(static_cast<char*>(ws->block) + 2 * up);
    ws->m = static_cast<int64_t>(m);
    s->space_ws = ws;
    return SCN_OK;
}

// out[t] for t < T: element elem[j] of in, with j the last entry of frame[] <= t;
// exact (repeat = 0): only when frame[j] == t; otherwise the fill element.
template <typename W>
__global__ void space_kernel(const W* in, int words, const int32_t* frame, const int32_t* elem, int64_t m, int64_t T,
                             int repeat, const W* fill, W* out) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < T;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int64_t lo = 0, hi = m;  // first index with frame > t
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (frame[mid] <= t) lo = mid + 1;
            else hi = mid;
        }
        const int64_t j = lo - 1;
        const bool have = j >= 0 && (repeat || frame[j] == t);
        const W* src = have ? in + static_cast<int64_t>(elem[j]) * words : fill;
        W* dst = out + t * words;
        for (int w = 0; w < words; ++w) dst[w] = src[w];
    }
}

// Slice starts of an n-element sequence: k starts a slice when k == 0 or
// flag[k] != 0.  One CTA walks the flags in tiles, each thread 8 elements,
// with a block-wide exclusive scan of the per-thread counts; starts come out
// in ascending order.
constexpr int kSliceThreads = 1024, kSlicePer = 8;

__global__ void __launch_bounds__(kSliceThreads) slice_kernel(const uint8_t* flag, int64_t n, int32_t* start,
                                                               int64_t* count) {
    __shared__ int warp_sum[32];
    __shared__ int64_t base_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < n; t0 += static_cast<int64_t>(kSliceThreads) * kSlicePer) {
        const int64_t k0 = t0 + static_cast<int64_t>(tid) * kSlicePer;
        uint32_t bits = 0;
#pragma unroll
        for (int i = 0; i < kSlicePer; ++i) {
            const int64_t k = k0 + i;
            if (k < n && (k == 0 || flag[k] != 0)) bits |= 1u << i;
        }
        const int c = __popc(bits);
        int incl = c;  // inclusive scan over the warp, then over warps
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int v = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            warp_sum[lane] = v;  // inclusive over warps
        }
        __syncthreads();
        const int64_t base = base_s;
        int64_t pos = base + (warp ? warp_sum[warp - 1] : 0) + incl - c;
#pragma unroll
        for (int i = 0; i < kSlicePer; ++i)
            if (bits & (1u << i)) start[pos++] = static_cast<int32_t>(k0 + i);
        __syncthreads();
        if (tid == kSliceThreads - 1) base_s = base + warp_sum[31];
        __syncthreads();
    }
    if (tid == 0) *count = base_s;
}

__global__ void slice_middles_kernel(const int32_t* start, const int64_t* count, int64_t n, int32_t* mid) {
    const int64_t m = *count;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t end = i + 1 < m ? start[i + 1] : n;
        mid[i] = static_cast<int32_t>((start[i] + end - 1) / 2);
    }
}

// Shot scores whose stencil stops at slice boundaries: score[k] = 0 where a
// slice starts (k == 0 or boundary[k] != 0), else the L1 distance of hist[k]
// and hist[k-1].  One warp per element.
__global__ void sliced_scores_kernel(const uint32_t* hist, int64_t n, int64_t pixel_count, const uint8_t* boundary,
                                     uint32_t* score, uint8_t* flag) {
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    if (k >= n) return;
    uint32_t d = 0;
    if (k > 0 && boundary[k] == 0) {
        const uint32_t* h = hist + k * 48;
        const uint32_t* g = h - 48;
        d = h[lane] > g[lane] ? h[lane] - g[lane] : g[lane] - h[lane];
        if (lane < 16) d += h[32 + lane] > g[32 + lane] ? h[32 + lane] - g[32 + lane] : g[32 + lane] - h[32 + lane];
    }
    const uint32_t s = __reduce_add_sync(0xffffffffu, d);
    if (lane == 0) {
        score[k] = s;
        flag[k] = (2ull * s > static_cast<uint64_t>(pixel_count)) ? 1 : 0;
    }
}

// Stencil S[a, b] shot score, one warp per output element k (global index): with
// P = -a frames before k and F = b + 1 frames from k, score = sum over the 48 bins
// of |F * sum_{j=a..-1} h[k+j] - P * sum_{j=0..b} h[k+j]|, flag = 2 score > P F px.
// Elements whose window leaves [0, n) or holds a slice start after its first
// frame score 0.  hist/boundary hold elements [first, first + count) only.
constexpr int kMaxWindow = 64;

__global__ void window_scores_kernel(const uint32_t* hist, const uint8_t* boundary, int64_t first, int64_t n, int a,
                                     int b, int64_t pixel_count, int64_t k0, int64_t k1, uint64_t* score,
                                     uint8_t* flag) {
    const int lane = threadIdx.x & 31;
    const int64_t k = k0 + blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    if (k >= k1) return;
    const int64_t P = -a, F = b + 1;
    bool zero = k + a < 0 || k + b >= n;
    if (!zero && boundary) {
        bool hit = false;
        for (int j = a + 1 + lane; j <= b; j += 32) hit |= boundary[k + j - first] != 0;
        zero = __any_sync(0xffffffffu, hit);
    }
    uint64_t d = 0;
    if (!zero) {
        for (int bin = lane; bin < 48; bin += 32) {
            int64_t before = 0, after = 0;
            for (int j = a; j < 0; ++j) before += hist[(k + j - first) * 48 + bin];
            for (int j = 0; j <= b; ++j) after += hist[(k + j - first) * 48 + bin];
            const int64_t v = F * before - P * after;
            d += static_cast<uint64_t>(v < 0 ? -v : v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) {
        score[k - k0] = d;
        flag[k - k0] = (2ull * d > static_cast<uint64_t>(P * F) * static_cast<uint64_t>(pixel_count)) ? 1 : 0;
    }
}

// Bounded-state shot score, one warp per run of outputs.  Run r has outputs
// [k0, k1) = [first + r*stride, first + r*stride + len) clipped to n, and
// processes elements max(0, k0 - warmup) .. k1 - 1 in order (the warmup).  The
// state is a reference histogram m (lane: bins lane and 32 + lane).  The first
// processed element, and a slice start, set m = h and output (0, 0); every
// other element outputs d = sum |h - m| and f = 2d > px, then sets m = h when f
// (a cut) else m += (h - m) >> shift (floor).  Histograms are read a block of
// kStateBlock elements ahead of the dependent chain.
constexpr int kStateBlock = 4;
constexpr int64_t kMaxStatePixels = 715827882;  // 6 * pixel_count < 2^32

__device__ __forceinline__ void state_load(const uint32_t* hist, const uint8_t* boundary, int64_t hfirst, int64_t j,
                                           int64_t k1, int lane, uint32_t (&h0)[kStateBlock],
                                           uint32_t (&h1)[kStateBlock], uint32_t (&bd)[kStateBlock]) {
#pragma unroll
    for (int u = 0; u < kStateBlock; ++u) {
        const int64_t e = j + u;
        h0[u] = 0;
        h1[u] = 0;
        bd[u] = 0;
        if (e < k1) {
            const uint32_t* row = hist + (e - hfirst) * 48;
            h0[u] = __ldg(row + lane);
            if (lane < 16) h1[u] = __ldg(row + 32 + lane);
            if (boundary) bd[u] = __ldg(boundary + (e - hfirst));
        }
    }
}

__global__ void bounded_state_kernel(const uint32_t* hist, const uint8_t* boundary, int64_t hfirst, int64_t n,
                                     int64_t pixel_count, int shift, int64_t warmup, int64_t first, int64_t len,
                                     int64_t stride, int64_t runs, uint32_t* score, uint8_t* flag) {
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    if (r >= runs) return;
    const int64_t k0 = first + r * stride;
    if (k0 >= n) return;
    const int64_t k1 = k0 + min(len, n - k0);
    const int64_t j0 = max(static_cast<int64_t>(0), k0 - warmup);
    const uint64_t px = static_cast<uint64_t>(pixel_count);
    uint32_t* out_s = score + r * len;  // element k goes to slot r*len + (k - k0)
    uint8_t* out_f = flag + r * len;
    int32_t m0 = 0, m1 = 0;
    uint32_t c0[kStateBlock], c1[kStateBlock], cb[kStateBlock];
    state_load(hist, boundary, hfirst, j0, k1, lane, c0, c1, cb);
    for (int64_t j = j0; j < k1; j += kStateBlock) {
        uint32_t n0[kStateBlock], n1[kStateBlock], nb[kStateBlock];
        state_load(hist, boundary, hfirst, j + kStateBlock, k1, lane, n0, n1, nb);
#pragma unroll
        for (int u = 0; u < kStateBlock; ++u) {
            const int64_t e = j + u;
            if (e >= k1) break;
            const int32_t h0 = static_cast<int32_t>(c0[u]), h1 = static_cast<int32_t>(c1[u]);
            uint32_t d = 0, f = 0;
            if (e == j0 || cb[u] != 0) {
                m0 = h0;
                m1 = h1;
            } else {
                const int32_t x0 = h0 - m0, x1 = h1 - m1;  // x1 = 0 on lanes >= 16
                d = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(abs(x0) + abs(x1)));
                f = 2ull * d > px ? 1u : 0u;
                if (f) {
                    m0 = h0;
                    m1 = h1;
                } else {
                    m0 += x0 >> shift;
                    m1 += x1 >> shift;
                }
            }
            if (lane == 0 && e >= k0) {
                out_s[e - k0] = d;
                out_f[e - k0] = static_cast<uint8_t>(f);
            }
        }
#pragma unroll
        for (int u = 0; u < kStateBlock; ++u) {
            c0[u] = n0[u];
            c1[u] = n1[u];
            cb[u] = nb[u];
        }
    }
}

// Montage: tile i (row-major over `cols` tiles) shows sequence element elem[i],
// nearest-neighbour downsampled: output pixel (x, y) of a tw x th tile takes
// source pixel (floor((2x+1) W / (2 tw)), floor((2y+1) H / (2 th))) of the
// BT.601 fixed-point RGB frame (chroma nearest).  Tiles past m, and tiles whose
// element is outside the sequence, are black.
__global__ void montage_kernel(const uint8_t* nv12, int64_t stride, int W, int H, const int32_t* slot, int64_t n,
                               const int32_t* elem, int64_t m, int cols, int tw, int th, int64_t out_w,
                               int64_t out_h, uint8_t* out) {
    const int64_t total = out_w * out_h;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < total;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t oy = p / out_w, ox = p - oy * out_w;
        const int64_t i = (oy / th) * cols + ox / tw;
        const int x = static_cast<int>(ox % tw), y = static_cast<int>(oy % th);
        uint8_t rgb[3] = {0, 0, 0};
        const int64_t e = i < m ? elem[i] : -1;
        if (e >= 0 && e < n) {
            const int sx = static_cast<int>(((2LL * x + 1) * W) / (2LL * tw));
            const int sy = static_cast<int>(((2LL * y + 1) * H) / (2LL * th));
            const uint8_t* f = nv12 + static_cast<int64_t>(slot[e]) * stride;
            const int C = static_cast<int>(f[static_cast<int64_t>(sy) * W + sx]) - 16;
            const uint8_t* uv = f + static_cast<int64_t>(W) * H + static_cast<int64_t>(sy >> 1) * W + (sx >> 1) * 2;
            const int D = static_cast<int>(uv[0]) - 128, E = static_cast<int>(uv[1]) - 128;
            const int r = (298 * C + 409 * E + 128) >> 8;
            const int g = (298 * C - 100 * D - 208 * E + 128) >> 8;
            const int b = (298 * C + 516 * D + 128) >> 8;
            rgb[0] = static_cast<uint8_t>(min(max(r, 0), 255));
            rgb[1] = static_cast<uint8_t>(min(max(g, 0), 255));
            rgb[2] = static_cast<uint8_t>(min(max(b, 0), 255));
        }
        out[3 * p] = rgb[0];
        out[3 * p + 1] = rgb[1];
        out[3 * p + 2] = rgb[2];
    }
}

int grid_for(int64_t work, int threads) {
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, sms * 8LL)));
}

}  // namespace

void free_space_workspace(scn_seq* s) {
    SpaceWs* ws = static_cast<SpaceWs*>(s->space_ws);
    if (!ws) return;
    obj_free(ws->block);
    delete ws;
    s->space_ws = nullptr;
}

}  // namespace scn

using namespace scn;

extern "C" {

scn_status scn_space(scn_seq* s, const void* d_in, int32_t elem_bytes, int32_t fill_mode, const void* h_fill,
                     void* d_out, void* stream) {
    if (!s || !d_out || elem_bytes < 1 || elem_bytes > kMaxElem) return SCN_EINVAL;
    if (fill_mode != SCN_FILL_VALUE && fill_mode != SCN_FILL_REPEAT) return SCN_EINVAL;
    if (s->n > 0 && !d_in) return SCN_EINVAL;
    const int64_t T = s->table->num_frames;
    if (T > 0x7fffffff) return SCN_ERANGE;
    SpaceWs* ws = nullptr;
    scn_status st = ensure_space_ws(s, ws);
    if (st != SCN_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (h_fill) SCN_CUDA_TRY(cudaMemcpyAsync(ws->fill, h_fill, elem_bytes, cudaMemcpyHostToDevice, cs));
    else SCN_CUDA_TRY(cudaMemsetAsync(ws->fill, 0, elem_bytes, cs));
    const bool words4 = elem_bytes % 4 == 0 && reinterpret_cast<uintptr_t>(d_in) % 4 == 0 &&
                        reinterpret_cast<uintptr_t>(d_out) % 4 == 0;
    const int g = grid_for(T, 256);
    if (words4)
        space_kernel<uint32_t><<<g, 256, 0, cs>>>(static_cast<const uint32_t*>(d_in), elem_bytes / 4, ws->frame,
                                                  ws->elem, ws->m, T, fill_mode == SCN_FILL_REPEAT,
                                                  reinterpret_cast<const uint32_t*>(ws->fill),
                                                  static_cast<uint32_t*>(d_out));
    else
        space_kernel<uint8_t><<<g, 256, 0, cs>>>(static_cast<const uint8_t*>(d_in), elem_bytes, ws->frame, ws->elem,
                                                 ws->m, T, fill_mode == SCN_FILL_REPEAT, ws->fill,
                                                 static_cast<uint8_t*>(d_out));
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

scn_status scn_slice(const uint8_t* d_flag, int64_t n, int32_t* d_start, int64_t* d_count, void* stream) {
    if (n < 0 || !d_count) return SCN_EINVAL;
    if (n > 0x7fffffff) return SCN_ERANGE;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        SCN_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), cs));
        return SCN_OK;
    }
    if (!d_flag || !d_start) return SCN_EINVAL;
    slice_kernel<<<1, kSliceThreads, 0, cs>>>(d_flag, n, d_start, d_count);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

scn_status scn_slice_middles(const int32_t* d_start, const int64_t* d_count, int64_t n, int32_t* d_mid, void* stream) {
    if (n < 0 || !d_count) return SCN_EINVAL;
    if (n == 0) return SCN_OK;
    if (!d_start || !d_mid) return SCN_EINVAL;
    slice_middles_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_start, d_count, n, d_mid);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

scn_status scn_shot_scores_sliced(const uint32_t* d_hist, int64_t n, int64_t pixel_count, const uint8_t* d_boundary,
                                  uint32_t* d_score, uint8_t* d_flag, void* stream) {
    if (n < 0 || pixel_count < 0) return SCN_EINVAL;
    if (n == 0) return SCN_OK;
    if (!d_hist || !d_boundary || !d_score || !d_flag) return SCN_EINVAL;
    const int64_t blocks = (n + 7) / 8;
    if (blocks > 0x7fffffff) return SCN_ERANGE;
    sliced_scores_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_hist, n, pixel_count, d_boundary, d_score, d_flag);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

scn_status scn_window_scores(const uint32_t* d_hist, int64_t hist_first, int64_t hist_count, int64_t n, int32_t a,
                             int32_t b, int64_t pixel_count, const uint8_t* d_boundary, int64_t k0, int64_t k1,
                             uint64_t* d_score, uint8_t* d_flag, void* stream) {
    if (a >= 0 || b < 0 || -a > kMaxWindow || b + 1 > kMaxWindow || pixel_count < 0 || n < 0) return SCN_EINVAL;
    if (k0 < 0 || k1 < k0 || k1 > n || hist_first < 0 || hist_count < 0) return SCN_ERANGE;
    if (k1 == k0) return SCN_OK;
    if (!d_hist || !d_score || !d_flag) return SCN_EINVAL;
    // dependency analysis: the outputs [k0, k1) read elements [k0 + a, k1 + b) within [0, n)
    const int64_t need0 = std::max<int64_t>(0, k0 + a), need1 = std::min<int64_t>(n, k1 + b);
    if (need0 < hist_first || need1 > hist_first + hist_count) return SCN_ERANGE;
    if (pixel_count > (int64_t(1) << 40)) return SCN_ERANGE;
    const int64_t blocks = (k1 - k0 + 7) / 8;
    if (blocks > 0x7fffffff) return SCN_ERANGE;
    window_scores_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_hist, d_boundary, hist_first, n, a, b, pixel_count, k0, k1, d_score, d_flag);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

scn_status scn_bounded_state_scores(const uint32_t* d_hist, int64_t hist_first, int64_t hist_count, int64_t n,
                                   int64_t pixel_count, int32_t shift, int64_t warmup, int64_t run_first,
                                   int64_t run_len, int64_t run_stride, int64_t runs, const uint8_t* d_boundary,
                                   uint32_t* d_score, uint8_t* d_flag, void* stream) {
    if (n < 0 || pixel_count < 0 || shift < 0 || shift > 30 || warmup < 0 || run_first < 0 || run_len < 1 ||
        run_stride < run_len || runs < 0 || hist_first < 0 || hist_count < 0)
        return SCN_EINVAL;
    if (pixel_count > kMaxStatePixels) return SCN_ERANGE;
    if (runs == 0 || run_first >= n) return SCN_OK;
    if (!d_hist || !d_score || !d_flag) return SCN_EINVAL;
    // the last run with outputs, and the dependency range of all runs (Sec. 4.2:
    // a warmup of W is the footprint i - W .. i)
    const int64_t r_last = std::min(runs - 1, (n - 1 - run_first) / run_stride);
    const int64_t need0 = std::max<int64_t>(0, run_first - warmup);
    const int64_t k_last = run_first + r_last * run_stride;  // < n
    const int64_t need1 = k_last + std::min(run_len, n - k_last);
    if (need0 < hist_first || need1 > hist_first + hist_count) return SCN_ERANGE;
    const int64_t blocks = (r_last + 1 + 7) / 8;
    if (blocks > 0x7fffffff) return SCN_ERANGE;
    bounded_state_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_hist, d_boundary, hist_first, n, pixel_count, shift, warmup, run_first, run_len, run_stride, r_last + 1,
        d_score, d_flag);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

scn_status scn_montage(const scn_seq* s, const int32_t* d_elem, int64_t m, int32_t cols, int32_t tile_w,
                       int32_t tile_h, uint8_t* d_out, void* stream) {
    if (!s || m < 0 || cols < 1 || tile_w < 1 || tile_h < 1 || tile_w > 4096 || tile_h > 4096) return SCN_EINVAL;
    if (m == 0) return SCN_OK;
    if (!d_elem || !d_out) return SCN_EINVAL;
    const int64_t rows = (m + cols - 1) / cols;
    const int64_t out_w = static_cast<int64_t>(cols) * tile_w, out_h = rows * tile_h;
    if (out_w * out_h > (int64_t(1) << 34)) return SCN_ERANGE;
    montage_kernel<<<grid_for(out_w * out_h, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        s->table->d_nv12, s->table->frame_stride, s->table->W, s->table->H, s->d_slot, s->n, d_elem, m, cols, tile_w,
        tile_h, out_w, out_h, d_out);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // extern "C"
