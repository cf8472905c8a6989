// Gated exact path: a cheap gate (the proposal network's logits, or any score)
// proposes candidate boundaries between consecutive sampled frames, and only
// the frames of proposed pairs go through the exact convert + histogram +
// score kernel, which keeps the final say: an unproposed pair gets score 0 and
// flag 0, a proposed pair gets its exact score and flag.
//
// Steps: proposals, compacted into a list of proposed elements k (pair k-1, k)
// with the storage slots of both frames of each -> one launch of the fused
// kernel over that 2m-element sequence, which writes each pair's score and flag
// to its element.  The kernels of a pass are launched as programmatic
// dependents of one another, so each one's launch overlaps its predecessor's end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "scn_internal.h"
#include "scn_ptx.cuh"

namespace scn {
namespace {

struct GateWs {
    void* block = nullptr;
    size_t bytes = 0;
    int64_t cap = 0;          // elements of the sequence it was made for
    int32_t* list = nullptr;  // [cap] proposed elements
    int32_t* slots2 = nullptr;  // [2 cap]
    uint32_t* hist2 = nullptr;  // [2 cap][48]
    uint32_t* partial = nullptr;  // [2 cap][48] (left zero)
    uint32_t* done = nullptr;
    uint32_t* pair = nullptr;
    uint32_t* queue = nullptr;
    int* status = nullptr;
    int* count = nullptr;
    // the cascade's prefiltered pairs: thumbnail indices, element, count
    int32_t* pre_prev = nullptr;
    int32_t* pre_cur = nullptr;
    int32_t* pre_elem = nullptr;
    int* pre_count = nullptr;
};

// Each proposed pair (k-1, k) is appended to the list together with the storage
// slots of its two frames, the 2m-element sequence the exact pass reads.  The
// count m stays on the device (*count), so no host round trip sits between the
// gate and the exact pass.
__global__ void propose_kernel(const float* gate, int64_t n, float tau, uint8_t* proposed, int32_t* list, int* count,
                               uint32_t* score, uint8_t* flag, const int32_t* slot, int32_t* slots2) {
    ptx::pdl_wait();
    ptx::pdl_release();
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const bool p = k >= 1 && gate[k] > tau;
        proposed[k] = p ? 1 : 0;
        score[k] = 0;
        flag[k] = 0;
        if (p) {
            const int i = atomicAdd(count, 1);
            list[i] = static_cast<int32_t>(k);
            slots2[2 * i] = slot[k - 1];
            slots2[2 * i + 1] = slot[k];
        }
    }
}

// Sum of |thumb[k] - thumb[k-1]| over the 2304 samples (0 for k = 0), by one
// warp: each lane takes 16-byte pieces of both thumbnails (4-byte pieces when
// the array is only 4-byte aligned); the total is in every lane.
__device__ __forceinline__ unsigned thumb_l1(const uint8_t* thumbs, int64_t k, int lane) {
    unsigned s = 0;
    if (k > 0) {
        if ((reinterpret_cast<uintptr_t>(thumbs) & 15u) == 0) {
            const uint4* a = reinterpret_cast<const uint4*>(thumbs + k * 2304);
            const uint4* b = reinterpret_cast<const uint4*>(thumbs + (k - 1) * 2304);
#pragma unroll
            for (int i = lane; i < 144; i += 32) {
                const uint4 x = a[i], y = b[i];
                s = __vsadu4(x.x, y.x) + __vsadu4(x.y, y.y) + __vsadu4(x.z, y.z) + __vsadu4(x.w, y.w) + s;
            }
        } else {
            const uint32_t* a = reinterpret_cast<const uint32_t*>(thumbs + k * 2304);
            const uint32_t* b = reinterpret_cast<const uint32_t*>(thumbs + (k - 1) * 2304);
            for (int i = lane; i < 576; i += 32) s = __vsadu4(a[i], b[i]) + s;
        }
    }
    return __reduce_add_sync(0xffffffffu, s);
}

// The luma + chroma gate of element k (0 for k = 0) by one warp: mean |dY| +
// mean |dU| + mean |dV| over two coarse YUV thumbnails (192 samples per plane,
// 576 bytes, 16-byte aligned), i.e. the sum of all 576 differences / 192.
__device__ __forceinline__ float yuv_gate(const uint8_t* yuv, int64_t k, int lane) {
    unsigned s = 0;
    if (k > 0 && lane < 36) {
        const uint4 x = reinterpret_cast<const uint4*>(yuv + k * 576)[lane];
        const uint4 y = reinterpret_cast<const uint4*>(yuv + (k - 1) * 576)[lane];
        s = __vsadu4(x.x, y.x) + __vsadu4(x.y, y.y) + __vsadu4(x.z, y.z) + __vsadu4(x.w, y.w);
    }
    if (k > 0 && lane < 4) {
        const uint4 x = reinterpret_cast<const uint4*>(yuv + k * 576)[32 + lane];
        const uint4 y = reinterpret_cast<const uint4*>(yuv + (k - 1) * 576)[32 + lane];
        s += __vsadu4(x.x, y.x) + __vsadu4(x.y, y.y) + __vsadu4(x.z, y.z) + __vsadu4(x.w, y.w);
    }
    return static_cast<float>(__reduce_add_sync(0xffffffffu, s)) / 192.f;
}

constexpr int kDiffWarps = 8;  // frames per 256-thread block, one warp each

// the luma gate (thumbs given) or the luma + chroma gate (yuv given) of every element (0 for k = 0)
__global__ void __launch_bounds__(32 * kDiffWarps) thumb_diff_kernel(const uint8_t* thumbs, const uint8_t* yuv,
                                                                     int64_t n, float* diff) {
    ptx::pdl_wait();
    ptx::pdl_release();
    const int64_t k = blockIdx.x * static_cast<int64_t>(kDiffWarps) + (threadIdx.x >> 5);
    if (k >= n) return;
    const int lane = threadIdx.x & 31;
    const float d = yuv ? yuv_gate(yuv, k, lane) : static_cast<float>(thumb_l1(thumbs, k, lane)) / 2304.f;
    if (lane == 0) diff[k] = d;
}

// Cascade prefilter, in the thumbnail-difference launch: d_diff[k] as
// thumb_diff_kernel writes it, every gate value set below any threshold, and
// each pair whose difference exceeds tau_diff listed for the network
// (thumbnail indices k-1, k, whose logit goes to gate element k).
__global__ void __launch_bounds__(32 * kDiffWarps) diff_prefilter_kernel(const uint8_t* yuv, int64_t n,
                                                                         float tau_diff, float* diff, float* gate,
                                                                         int32_t* prev, int32_t* cur, int32_t* elem,
                                                                         int* count, int* zero) {
    ptx::pdl_wait();
    ptx::pdl_release();
    // the proposal list's counter, appended to by the gate after the network
    if (blockIdx.x == 0 && threadIdx.x == 0) *zero = 0;
    const int64_t k = blockIdx.x * static_cast<int64_t>(kDiffWarps) + (threadIdx.x >> 5);
    if (k >= n) return;
    const float dk = yuv_gate(yuv, k, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) {
        diff[k] = dk;
        gate[k] = -INFINITY;
        if (k > 0 && dk > tau_diff) {
            const int i = atomicAdd(count, 1);
            prev[i] = static_cast<int32_t>(k - 1);
            cur[i] = static_cast<int32_t>(k);
            elem[i] = static_cast<int32_t>(k);
        }
    }
}

scn_status ensure_ws(scn_seq* s, GateWs*& ws) {
    ws = static_cast<GateWs*>(s->gate_ws);
    if (ws && ws->cap >= s->n) return SCN_OK;
    if (ws) {
        obj_free(ws->block);
        delete ws;
        s->gate_ws = nullptr;
    }
    ws = new (std::nothrow) GateWs;
    if (!ws) return SCN_ENOMEM;
    const int64_t c = std::max<int64_t>(s->n, 1);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t parts[] = {up(c * 4), up(2 * c * 4), up(2 * c * 48 * 4), up(2 * c * 48 * 4), up(2 * c * 4),
                            up(2 * c * 4), 256, 256, 256, up(c * 4), up(c * 4), up(c * 4), 256};
    size_t total = 0;
    for (size_t p : parts) total += p;
    cudaError_t e = obj_alloc(&ws->block, total);
    if (e == cudaSuccess) e = obj_zero(ws->block, total);
    if (e == cudaSuccess) e = obj_finish();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        obj_free(ws->block);
        delete ws;
        ws = nullptr;
        return SCN_ECUDA;
    }
    char* p = static_cast<char*>(ws->block);
    void** dst[] = {reinterpret_cast<void**>(&ws->list),    reinterpret_cast<void**>(&ws->slots2),
                    reinterpret_cast<void**>(&ws->hist2),   reinterpret_cast<void**>(&ws->partial),
                    reinterpret_cast<void**>(&ws->done),    reinterpret_cast<void**>(&ws->pair),
                    reinterpret_cast<void**>(&ws->queue),   reinterpret_cast<void**>(&ws->status),
                    reinterpret_cast<void**>(&ws->count),   reinterpret_cast<void**>(&ws->pre_prev),
                    reinterpret_cast<void**>(&ws->pre_cur), reinterpret_cast<void**>(&ws->pre_elem),
                    reinterpret_cast<void**>(&ws->pre_count)};
    static_assert(sizeof(parts) / sizeof(parts[0]) == sizeof(dst) / sizeof(dst[0]), "workspace parts");
    for (size_t i = 0; i < sizeof(parts) / sizeof(parts[0]); ++i) {
        *dst[i] = p;
        p += parts[i];
    }
    ws->cap = c;
    ws->bytes = total;
    s->gate_ws = ws;
    return SCN_OK;
}

// The gate, then the exact kernel on the proposed pairs.  count_zeroed: an
// earlier kernel of the same pass has already zeroed the list's counter.
scn_status gated_hist(scn_seq* s, const float* d_gate, float tau, uint8_t* d_proposed, uint32_t* d_score,
                      uint8_t* d_flag, int64_t* h_nproposed, cudaStream_t cs, bool count_zeroed) {
    if (!s || !d_gate || !d_proposed || !d_score || !d_flag) return SCN_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_score) & 3u) return SCN_EINVAL;
    if (h_nproposed) *h_nproposed = 0;
    if (s->n == 0) return SCN_OK;
    GateWs* ws = nullptr;
    scn_status st = ensure_ws(s, ws);
    if (st != SCN_OK) return st;
    if (!count_zeroed) SCN_CUDA_TRY(cudaMemsetAsync(ws->count, 0, sizeof(int), cs));
    const int64_t blocks = std::min<int64_t>((s->n + 255) / 256, 148 * 8);
    SCN_CUDA_TRY(launch_pdl(propose_kernel, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, cs, d_gate, s->n, tau,
                            d_proposed, ws->list, ws->count, d_score, d_flag,
                            static_cast<const int32_t*>(s->d_slot), ws->slots2));
    // m = *ws->count stays on the device: the exact launch is sized for the
    // largest m (n - 1 pairs) and reads m itself
    const int64_t cap = s->n;
    // the exact kernel over the 2m frames of the proposed pairs: one contiguous
    // range of row pairs per CTA, each CTA computing its range from m on the device;
    // the score of pair i (elements 2i, 2i + 1) goes straight to element list[i]
    scn_seq q;
    q.table = s->table;
    q.n = 2 * cap;
    q.tune = s->tune;
    HistShape sh = resolve_hist_shape(&q);
    const int W = s->table->W, H = s->table->H;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    sh.grid = s->tune.grid > 0 ? s->tune.grid : sms;
    sh.rp_per_cta = -1;
    sh.item_rp = static_cast<int>(std::min<int64_t>(H / 2, std::max<int64_t>(1, kItemPixelsMax / (2LL * W))));
    Launch L = single_launch(s->table, q.n, ws->slots2, sh);
    L.d_count = ws->count;
    L.count_mul = 2;
    L.job0.hist = ws->hist2;
    L.job0.score = d_score;
    L.job0.flag = d_flag;
    L.job0.score_at = ws->list;
    L.job0.partial = ws->partial;
    L.job0.done = ws->done;
    L.job0.pair = ws->pair;
    L.queue = ws->queue;
    L.status = s->d_status;
    st = launch_hist(L, cs);
    if (st != SCN_OK) return st;
    if (h_nproposed) {  // the only host wait, at the end and only when asked for
        int m = 0;
        SCN_CUDA_TRY(cudaMemcpyAsync(&m, ws->count, sizeof(int), cudaMemcpyDeviceToHost, cs));
        SCN_CUDA_TRY(cudaStreamSynchronize(cs));
        *h_nproposed = m;
    }
    return SCN_OK;
}

}  // namespace

cudaError_t reset_gate_workspace(scn_seq* s, cudaStream_t st) {
    GateWs* ws = static_cast<GateWs*>(s->gate_ws);
    if (!ws) return cudaSuccess;
    // everything in the block is scratch of one call: zero all of it
    return cudaMemsetAsync(ws->block, 0, ws->bytes, st);
}

void free_gate_workspace(scn_seq* s) {
    GateWs* ws = static_cast<GateWs*>(s->gate_ws);
    if (!ws) return;
    obj_free(ws->block);
    delete ws;
    s->gate_ws = nullptr;
}

}  // namespace scn

using namespace scn;

extern "C" {

scn_status scn_thumb_diff(const uint8_t* d_thumbs, int64_t n, float* d_diff, void* stream) {
    if (n < 0) return SCN_EINVAL;
    if (n == 0) return SCN_OK;
    if (!d_thumbs || !d_diff || (reinterpret_cast<uintptr_t>(d_thumbs) & 3u)) return SCN_EINVAL;
    if (n > 0x7fffffff) return SCN_ERANGE;
    SCN_CUDA_TRY(launch_pdl(thumb_diff_kernel, dim3(static_cast<unsigned>((n + kDiffWarps - 1) / kDiffWarps)),
                            dim3(32 * kDiffWarps), 0, static_cast<cudaStream_t>(stream), static_cast<const uint8_t*>(d_thumbs),
                            static_cast<const uint8_t*>(nullptr), n, d_diff));
    return SCN_OK;
}

scn_status scn_thumb_diff_yuv(const uint8_t* d_yuv, int64_t n, float* d_diff, void* stream) {
    if (n < 0) return SCN_EINVAL;
    if (n == 0) return SCN_OK;
    if (!d_yuv || !d_diff || (reinterpret_cast<uintptr_t>(d_yuv) & 15u)) return SCN_EINVAL;
    if (n > 0x7fffffff) return SCN_ERANGE;
    SCN_CUDA_TRY(launch_pdl(thumb_diff_kernel, dim3(static_cast<unsigned>((n + kDiffWarps - 1) / kDiffWarps)),
                            dim3(32 * kDiffWarps), 0, static_cast<cudaStream_t>(stream), static_cast<const uint8_t*>(nullptr),
                            static_cast<const uint8_t*>(d_yuv), n, d_diff));
    return SCN_OK;
}

scn_status scn_gated_hist_scores(scn_seq* s, const float* d_gate, float tau, uint8_t* d_proposed, uint32_t* d_score,
                                 uint8_t* d_flag, int64_t* h_nproposed, void* stream) {
    return gated_hist(s, d_gate, tau, d_proposed, d_score, d_flag, h_nproposed, static_cast<cudaStream_t>(stream),
                      false);
}

scn_status scn_proposal_hist_scores(scn_seq* s, scn_cnn* net, float tau, uint8_t* d_thumbs, float* d_logits,
                                    uint8_t* d_proposed, uint32_t* d_score, uint8_t* d_flag, int64_t* h_nproposed,
                                    void* stream) {
    if (!s || !net || !d_thumbs || !d_logits) return SCN_EINVAL;
    if (h_nproposed) *h_nproposed = 0;
    if (s->n == 0) return SCN_OK;
    GateWs* ws = nullptr;
    scn_status st = ensure_ws(s, ws);
    if (st != SCN_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // the thumbnail launch also zeroes the proposal list's counter
    st = launch_thumbs(s, d_thumbs, nullptr, ws->count, cs);
    if (st != SCN_OK) return st;
    if (s->n > 1) {
        // pair (k-1, k) -> logit k
        st = scn_cnn_forward(net, d_thumbs, nullptr, nullptr, s->n - 1, d_logits + 1, stream);
        if (st != SCN_OK) return st;
    }
    return gated_hist(s, d_logits, tau, d_proposed, d_score, d_flag, h_nproposed, cs, true);
}


scn_status scn_cascade_hist_scores(scn_seq* s, scn_cnn* net, float tau_diff, float tau_net, uint8_t* d_thumbs,
                                   uint8_t* d_yuv, float* d_diff, float* d_gate, uint8_t* d_proposed,
                                   uint32_t* d_score, uint8_t* d_flag, int64_t* h_nproposed, void* stream) {
    if (!s || !net || !d_thumbs || !d_yuv || !d_diff || !d_gate || !d_proposed || !d_score || !d_flag)
        return SCN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_thumbs) & 15u) || (reinterpret_cast<uintptr_t>(d_yuv) & 15u)) return SCN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_diff) | reinterpret_cast<uintptr_t>(d_gate)) & 3u) return SCN_EINVAL;
    if (h_nproposed) *h_nproposed = 0;
    if (s->n == 0) return SCN_OK;
    if (s->n > 0x7fffffff) return SCN_ERANGE;
    GateWs* ws = nullptr;
    scn_status st = ensure_ws(s, ws);
    if (st != SCN_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // coarse YUV thumbnails of every frame (the gate's input), not the luma thumbnails;
    // the launch zeroes the prefilter's counter, the prefilter the proposal list's
    st = launch_thumbs(s, nullptr, d_yuv, ws->pre_count, cs);
    if (st != SCN_OK) return st;
    SCN_CUDA_TRY(launch_pdl(diff_prefilter_kernel, dim3(static_cast<unsigned>((s->n + kDiffWarps - 1) / kDiffWarps)),
                            dim3(32 * kDiffWarps), 0, cs, static_cast<const uint8_t*>(d_yuv), s->n, tau_diff, d_diff,
                            d_gate, ws->pre_prev, ws->pre_cur, ws->pre_elem, ws->pre_count, ws->count));
    if (s->n > 1) {
        // luma thumbnails only for the frames of the listed pairs: what the network reads
        st = launch_thumbs_listed(s, ws->pre_prev, ws->pre_cur, ws->pre_count, s->n - 1, d_thumbs, cs);
        if (st != SCN_OK) return st;
        // the network only on the listed pairs (the launch is sized for all n-1 and reads the
        // count); the logit of listed pair i goes straight to d_gate[elem[i]]
        st = cnn_forward_counted(net, d_thumbs, ws->pre_prev, ws->pre_cur, s->n - 1, ws->pre_count, d_gate, cs,
                                 ws->pre_elem);
        if (st != SCN_OK) return st;
    }
    return gated_hist(s, d_gate, tau_net, d_proposed, d_score, d_flag, h_nproposed, cs, true);
}

}  // extern "C"
