// Map ops over a sampled sequence: bilinear resize + normalisation of the RGB
// frame (the "Resize" stage ahead of a network, Sec. 3.1 and Sec. 5.1.2), and
// subsampled luma thumbnails.
//
// Resize definition (half-pixel centres, source index clamped at 0, upper
// neighbour clamped to the last row / column, no antialias, stretch):
//   sy = max((oy + 0.5) * H / oh - 0.5, 0), y0 = floor(sy), y1 = min(y0 + 1, H - 1),
//   ly = sy - y0 (same for x); v = (1-ly)((1-lx)P00 + lx P01) + ly((1-lx)P10 + lx P11)
//   out[c][oy][ox] = (v / 255 - mean[c]) / std[c]
// on the BT.601 fixed-point RGB of each source pixel.  The source coordinate is
// the rational ((2o+1)*S - O) / (2*O): its floor and the fraction's numerator
// come from integer arithmetic, the horizontal step is exact in integers, and
// only the vertical step and the normalisation round (in fp32).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "scn_internal.h"
#include "scn_ptx.cuh"

namespace scn {
namespace {

struct ResizeArgs {
    const uint8_t* nv12;
    int64_t stride;
    int W, H;
    const int32_t* slot;
    int oh, ow;
    float scale[3], bias[3];  // out = V * scale + bias: scale = 1/(255 std dx dy), bias = -mean/std
    float* out32;            // [n][3][oh][ow] FP32, or null
    __nv_bfloat16* out16;    // [n][3][oh][ow] BF16 (RNE of the FP32 value), or null
};

// Source tap of output index o (size O) in a source of size S: first index i0
// and weight numerator r of the second one, over the denominator 2 O.
__device__ __forceinline__ void src_tap(int o, int S, int O, int& i0, int& r) {
    const int num = (2 * o + 1) * S - O;
    if (num <= 0) {
        i0 = 0;
        r = 0;
    } else {
        i0 = num / (2 * O);
        r = num - i0 * (2 * O);
    }
}

// BT.601 fixed-point RGB of luma Y with the chroma word uv (U in byte 0, V in byte 1)
__device__ __forceinline__ void rgb601(int Y, uint32_t uv, int (&p)[3]) {
    const int C = 298 * Y - 4640;  // 298 (Y - 16) + 128
    const int D = static_cast<int>(uv & 0xFFu) - 128, E = static_cast<int>(uv >> 8) - 128;
    p[0] = min(max((C + 409 * E) >> 8, 0), 255);
    p[1] = min(max((C - 100 * D - 208 * E) >> 8, 0), 255);
    p[2] = min(max((C + 516 * D) >> 8, 0), 255);
}

// v as fp32, exactly, for 0 <= v < 2^23: v in the mantissa of 2^23, minus 2^23
__device__ __forceinline__ float small_to_float(int v) { return __int_as_float(v | 0x4B000000) - 8388608.f; }

// One CTA per 32 x 32 output tile of one element: the tile's source columns and
// rows are computed once into shared memory; thread (lane, warp) produces column
// lane of rows warp, warp + 8, warp + 16, warp + 24.  With dx = 2 ow, dy = 2 oh:
//   top = (dx - rx) P00 + rx P01, bottom = (dx - rx) P10 + rx P11   (exact integers < 2^23)
//   V = (dy - ry) top + ry bottom = dx dy v,  out = V * scale + bias
constexpr int kRzTile = 32;

__global__ void __launch_bounds__(256) resize_kernel(ResizeArgs a) {
    ptx::pdl_wait();  // launched as a programmatic dependent: global memory only after the wait
    ptx::pdl_release();
    __shared__ int2 tap[2 * kRzTile];  // columns, then rows: (first index, weight numerator)
    const int k = blockIdx.z, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ox0 = blockIdx.x * kRzTile, oy0 = blockIdx.y * kRzTile;
    if (tid < 2 * kRzTile) {
        int i0, r;
        if (tid < kRzTile)
            src_tap(min(ox0 + tid, a.ow - 1), a.W, a.ow, i0, r);
        else
            src_tap(min(oy0 + tid - kRzTile, a.oh - 1), a.H, a.oh, i0, r);
        tap[tid] = make_int2(i0, r);
    }
    __syncthreads();
    const int ox = ox0 + lane;
    if (ox >= a.ow) return;
    const uint8_t* f = a.nv12 + static_cast<int64_t>(a.slot[k]) * a.stride;
    const uint8_t* uvp = f + static_cast<int64_t>(a.W) * a.H;
    const int x0 = tap[lane].x, x1 = min(x0 + 1, a.W - 1), rx = tap[lane].y;
    const int cx0 = x0 & ~1, cx1 = x1 & ~1;
    const int wx0 = 2 * a.ow - rx;
    const int64_t npix = static_cast<int64_t>(a.oh) * a.ow;
    const int64_t base = static_cast<int64_t>(k) * 3 * npix + ox;
    for (int j = warp; j < kRzTile; j += 8) {
        const int oy = oy0 + j;
        if (oy >= a.oh) break;
        const int y0 = tap[kRzTile + j].x, y1 = min(y0 + 1, a.H - 1), ry = tap[kRzTile + j].y;
        const uint8_t* l0 = f + static_cast<int64_t>(y0) * a.W;
        const uint8_t* l1 = f + static_cast<int64_t>(y1) * a.W;
        const uint8_t* c0 = uvp + static_cast<int64_t>(y0 >> 1) * a.W;
        const uint8_t* c1 = uvp + static_cast<int64_t>(y1 >> 1) * a.W;
        int p00[3], p01[3], p10[3], p11[3];
        rgb601(__ldg(l0 + x0), __ldg(reinterpret_cast<const uint16_t*>(c0 + cx0)), p00);
        rgb601(__ldg(l0 + x1), __ldg(reinterpret_cast<const uint16_t*>(c0 + cx1)), p01);
        rgb601(__ldg(l1 + x0), __ldg(reinterpret_cast<const uint16_t*>(c1 + cx0)), p10);
        rgb601(__ldg(l1 + x1), __ldg(reinterpret_cast<const uint16_t*>(c1 + cx1)), p11);
        const float wy0 = static_cast<float>(2 * a.oh - ry), wy1 = static_cast<float>(ry);
        const int64_t o = base + static_cast<int64_t>(oy) * a.ow;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int top = wx0 * p00[c] + rx * p01[c];
            const int bot = wx0 * p10[c] + rx * p11[c];
            const float V = fmaf(wy0, small_to_float(top), wy1 * small_to_float(bot));
            const float out = fmaf(V, a.scale[c], a.bias[c]);
            if (a.out32) a.out32[o + c * npix] = out;
            if (a.out16) a.out16[o + c * npix] = __float2bfloat16_rn(out);
        }
    }
}

// Thumbnail gathers: every sample is its own 32-byte sector request, so a
// thread issues all of its loads before its first store (byte pointers may
// alias, which would otherwise keep each load behind the previous store).
constexpr int kThumbThreads = 192;  // 2304 = 12 x 192 luma samples; 192 coarse samples per plane

// Luma thumbnail of one frame f into o: o[r][c] = Y[s r][s c], 12 samples per thread.
__device__ __forceinline__ void luma_thumb(const uint8_t* __restrict__ f, int W, int s, uint8_t* __restrict__ o) {
    uint8_t v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const int i = threadIdx.x + q * kThumbThreads, r = i >> 6, c = i & 63;
        v[q] = __ldg(f + static_cast<int64_t>(s * r) * W + s * c);
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) o[threadIdx.x + q * kThumbThreads] = v[q];
}

// One block per frame: the luma thumbnail out[k] (when out is given) and the
// coarse YUV thumbnail (when yuv is given): yuv[k][0][r][c] = Y[6 s r][2 s c],
// yuv[k][1..2][r][c] = U, V of chroma sample (s c, 3 s r), the one under that
// luma pixel (one 16-bit load for both), r < 6, c < 32.  The gather's cost is
// the 128-byte lines it touches, so the coarse thumbnail samples 6 luma rows
// and 6 chroma rows (180 lines of a 1080p frame against 540 for the luma
// thumbnail).
__global__ void __launch_bounds__(kThumbThreads) thumbs_kernel(const uint8_t* __restrict__ nv12, int64_t stride, int W,
                                                              int H, int s, const int32_t* __restrict__ slot,
                                                              uint8_t* __restrict__ out, uint8_t* __restrict__ yuv,
                                                              int* zero) {
    ptx::pdl_wait();
    ptx::pdl_release();
    const int k = blockIdx.x;
    // a counter the next kernels of a proposal pass append to, zeroed here instead of by a
    // separate memset (every earlier reader of it has completed before pdl_wait returned)
    if (zero && k == 0 && threadIdx.x == 0) *zero = 0;
    const uint8_t* f = nv12 + static_cast<int64_t>(slot[k]) * stride;
    if (out) luma_thumb(f, W, s, out + static_cast<int64_t>(k) * 2304);
    if (yuv) {
        const uint8_t* plane = f + static_cast<int64_t>(W) * H;
        const int i = threadIdx.x, r = i >> 5, c = i & 31;  // 192 threads = 6 x 32 samples
        const uint8_t y = __ldg(f + static_cast<int64_t>(6 * s * r) * W + 2 * s * c);
        const uint16_t w = __ldg(reinterpret_cast<const uint16_t*>(plane + static_cast<int64_t>(3 * s * r) * W + 2 * s * c));
        uint8_t* o = yuv + static_cast<int64_t>(k) * 576;
        o[i] = y;
        o[192 + i] = static_cast<uint8_t>(w & 0xFF);
        o[384 + i] = static_cast<uint8_t>(w >> 8);
    }
}

// Luma thumbnails of the two frames of each listed pair i < *count (elements
// prev[i] and cur[i] of the sequence) into out[element]; a frame shared by two
// listed pairs is written twice with the same bytes.  One block per frame of a
// listed pair (block 2i + q), grid-stride over them.
__global__ void __launch_bounds__(kThumbThreads) thumbs_listed_kernel(const uint8_t* __restrict__ nv12, int64_t stride,
                                                                     int W, int s, const int32_t* __restrict__ slot,
                                                                     const int32_t* __restrict__ prev,
                                                                     const int32_t* __restrict__ cur,
                                                                     const int* __restrict__ count,
                                                                     uint8_t* __restrict__ out) {
    ptx::pdl_wait();
    ptx::pdl_release();
    const int64_t m2 = 2 * static_cast<int64_t>(*count);
    for (int64_t j = blockIdx.x; j < m2; j += gridDim.x) {
        const int32_t k = (j & 1) ? cur[j >> 1] : prev[j >> 1];
        luma_thumb(nv12 + static_cast<int64_t>(slot[k]) * stride, W, s, out + static_cast<int64_t>(k) * 2304);
    }
}

}  // namespace

scn_status launch_thumbs(const scn_seq* s, uint8_t* d_thumb, uint8_t* d_yuv, int* zero, cudaStream_t st) {
    if (!s || (!d_thumb && !d_yuv)) return SCN_EINVAL;
    const int W = s->table->W, H = s->table->H;
    if (W % 64 || H % 36 || W / 64 != H / 36) return SCN_EUNSUPPORTED;
    if (s->n == 0) return SCN_OK;
    if (s->n > 0x7fffffff) return SCN_ERANGE;
    SCN_CUDA_TRY(launch_pdl(thumbs_kernel, dim3(static_cast<unsigned>(s->n)), dim3(kThumbThreads), 0, st,
                            s->table->d_nv12, s->table->frame_stride, W, H, W / 64,
                            static_cast<const int32_t*>(s->d_slot), d_thumb, d_yuv, zero));
    return SCN_OK;
}
}  // namespace scn



namespace scn {
namespace {
scn_status launch_resize(scn_seq* s, int32_t oh, int32_t ow, const float* h_mean, const float* h_std, float* out32,
                         __nv_bfloat16* out16, void* stream) {
    if (oh > 16384 || ow > 16384) return SCN_ERANGE;  // keeps (2o+1)*S in int32
    for (int c = 0; c < 3; ++c)
        if (!(h_std[c] != 0.f)) return SCN_EINVAL;
    if (s->n == 0) return SCN_OK;
    if (s->n > 65535) return SCN_ERANGE;  // one grid z index per element
    ResizeArgs a;
    a.nv12 = s->table->d_nv12;
    a.stride = s->table->frame_stride;
    a.W = s->table->W;
    a.H = s->table->H;
    a.slot = s->d_slot;
    a.oh = oh;
    a.ow = ow;
    const double dxdy = 4.0 * static_cast<double>(oh) * static_cast<double>(ow);
    for (int c = 0; c < 3; ++c) {
        a.scale[c] = static_cast<float>(1.0 / (255.0 * static_cast<double>(h_std[c]) * dxdy));
        a.bias[c] = static_cast<float>(-static_cast<double>(h_mean[c]) / static_cast<double>(h_std[c]));
    }
    a.out32 = out32;
    a.out16 = out16;
    dim3 grid((ow + kRzTile - 1) / kRzTile, (oh + kRzTile - 1) / kRzTile, static_cast<unsigned>(s->n));
    SCN_CUDA_TRY(launch_pdl(resize_kernel, grid, dim3(256), 0, static_cast<cudaStream_t>(stream), a));
    return SCN_OK;
}
}  // namespace
}  // namespace scn

namespace scn {
scn_status launch_thumbs_listed(const scn_seq* s, const int32_t* prev, const int32_t* cur, const int* count,
                                int64_t max_pairs, uint8_t* out, cudaStream_t st) {
    const int W = s->table->W, H = s->table->H;
    if (W % 64 || H % 36 || W / 64 != H / 36) return SCN_EUNSUPPORTED;
    if (max_pairs <= 0) return SCN_OK;
    // one block per listed frame, sized for the common case (a prefilter that passes a few
    // percent of the pairs); more listed frames loop over the same blocks
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>(2 * max_pairs, 4LL * sms));
    SCN_CUDA_TRY(launch_pdl(thumbs_listed_kernel, dim3(grid), dim3(kThumbThreads), 0, st, s->table->d_nv12,
                            s->table->frame_stride, W, W / 64, static_cast<const int32_t*>(s->d_slot), prev, cur,
                            count, out));
    return SCN_OK;
}
}  // namespace scn

extern "C" {

scn_status scn_resize_norm(scn_seq* s, int32_t oh, int32_t ow, const float* h_mean, const float* h_std, int32_t dtype,
                           void* d_out, void* stream) {
    if (!s || !h_mean || !h_std || !d_out || oh < 1 || ow < 1) return SCN_EINVAL;
    if (dtype != SCN_F32 && dtype != SCN_BF16) return SCN_EINVAL;
    const uintptr_t al = dtype == SCN_F32 ? 3u : 1u;
    if (reinterpret_cast<uintptr_t>(d_out) & al) return SCN_EINVAL;
    return scn::launch_resize(s, oh, ow, h_mean, h_std, dtype == SCN_F32 ? static_cast<float*>(d_out) : nullptr,
                              dtype == SCN_BF16 ? static_cast<__nv_bfloat16*>(d_out) : nullptr, stream);
}

scn_status scn_resize_norm_both(scn_seq* s, int32_t oh, int32_t ow, const float* h_mean, const float* h_std,
                                float* d_out_f32, void* d_out_bf16, void* stream) {
    if (!s || !h_mean || !h_std || !d_out_f32 || !d_out_bf16 || oh < 1 || ow < 1) return SCN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_out_f32) & 3u) || (reinterpret_cast<uintptr_t>(d_out_bf16) & 1u))
        return SCN_EINVAL;
    return scn::launch_resize(s, oh, ow, h_mean, h_std, d_out_f32, static_cast<__nv_bfloat16*>(d_out_bf16), stream);
}

scn_status scn_thumbs_yuv(scn_seq* s, uint8_t* d_thumb, uint8_t* d_yuv, void* stream) {
    return scn::launch_thumbs(s, d_thumb, d_yuv, nullptr, static_cast<cudaStream_t>(stream));
}

scn_status scn_thumbs(scn_seq* s, uint8_t* d_thumb, void* stream) {
    if (!d_thumb) return SCN_EINVAL;
    return scn_thumbs_yuv(s, d_thumb, nullptr, stream);
}

}  // extern "C"
