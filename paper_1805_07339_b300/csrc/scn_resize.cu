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
// the rational ((2o+1)*S - O) / (2*O); floor and fraction come from exact
// integer arithmetic so the weights carry a single fp32 rounding.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "scn_internal.h"

namespace scn {
namespace {

struct ResizeArgs {
    const uint8_t* nv12;
    int64_t stride;
    int W, H;
    const int32_t* slot;
    int oh, ow;
    float scale[3], bias[3];  // out = v * scale + bias, scale = 1/(255 std), bias = -mean/std
    float inv255;
    float mean[3], istd[3];
    float* out32;            // [n][3][oh][ow] FP32, or null
    __nv_bfloat16* out16;    // [n][3][oh][ow] BF16 (RNE of the FP32 value), or null
};

__device__ __forceinline__ void src_coord(int o, int S, int O, int& i0, int& i1, float& l) {
    const int num = (2 * o + 1) * S - O;
    if (num <= 0) {
        i0 = 0;
        l = 0.f;
    } else {
        const int den = 2 * O;
        i0 = num / den;
        l = static_cast<float>(num - i0 * den) / static_cast<float>(den);
    }
    i1 = min(i0 + 1, S - 1);
}

__device__ __forceinline__ void rgb_at(const uint8_t* f, int W, int H, int x, int y, int rgb[3]) {
    const int Y = __ldg(f + static_cast<int64_t>(y) * W + x);
    const uint8_t* uv = f + static_cast<int64_t>(W) * H + static_cast<int64_t>(y >> 1) * W + (x & ~1);
    const int U = __ldg(uv), V = __ldg(uv + 1);
    const int C = 298 * (Y - 16) + 128, D = U - 128, E = V - 128;
    rgb[0] = min(max((C + 409 * E) >> 8, 0), 255);
    rgb[1] = min(max((C - 100 * D - 208 * E) >> 8, 0), 255);
    rgb[2] = min(max((C + 516 * D) >> 8, 0), 255);
}

__global__ void __launch_bounds__(256) resize_kernel(ResizeArgs a) {
    const int k = blockIdx.y;
    const int npix = a.oh * a.ow;
    const uint8_t* f = a.nv12 + static_cast<int64_t>(a.slot[k]) * a.stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        const int oy = i / a.ow, ox = i - oy * a.ow;
        int y0, y1, x0, x1;
        float ly, lx;
        src_coord(oy, a.H, a.oh, y0, y1, ly);
        src_coord(ox, a.W, a.ow, x0, x1, lx);
        int p00[3], p01[3], p10[3], p11[3];
        rgb_at(f, a.W, a.H, x0, y0, p00);
        rgb_at(f, a.W, a.H, x1, y0, p01);
        rgb_at(f, a.W, a.H, x0, y1, p10);
        rgb_at(f, a.W, a.H, x1, y1, p11);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float top = (1.f - lx) * static_cast<float>(p00[c]) + lx * static_cast<float>(p01[c]);
            const float bot = (1.f - lx) * static_cast<float>(p10[c]) + lx * static_cast<float>(p11[c]);
            const float v = (1.f - ly) * top + ly * bot;
            const float o = (v * a.inv255 - a.mean[c]) * a.istd[c];
            const int64_t idx = (static_cast<int64_t>(k) * 3 + c) * npix + i;
            if (a.out32) a.out32[idx] = o;
            if (a.out16) a.out16[idx] = __float2bfloat16_rn(o);
        }
    }
}

__global__ void __launch_bounds__(256) thumbs_kernel(const uint8_t* nv12, int64_t stride, int W, int s,
                                                    const int32_t* slot, uint8_t* out) {
    const int k = blockIdx.x;
    const uint8_t* f = nv12 + static_cast<int64_t>(slot[k]) * stride;
    for (int i = threadIdx.x; i < 36 * 64; i += blockDim.x) {
        const int r = i >> 6, c = i & 63;
        out[static_cast<int64_t>(k) * 2304 + i] = __ldg(f + static_cast<int64_t>(s * r) * W + s * c);
    }
}

}  // namespace
}  // namespace scn



namespace scn {
namespace {
scn_status launch_resize(scn_seq* s, int32_t oh, int32_t ow, const float* h_mean, const float* h_std, float* out32,
                         __nv_bfloat16* out16, void* stream) {
    if (oh > 16384 || ow > 16384) return SCN_ERANGE;  // keeps (2o+1)*S in int32
    for (int c = 0; c < 3; ++c)
        if (!(h_std[c] != 0.f)) return SCN_EINVAL;
    if (s->n == 0) return SCN_OK;
    if (s->n > 65535) return SCN_ERANGE;  // one grid row per element
    ResizeArgs a;
    a.nv12 = s->table->d_nv12;
    a.stride = s->table->frame_stride;
    a.W = s->table->W;
    a.H = s->table->H;
    a.slot = s->d_slot;
    a.oh = oh;
    a.ow = ow;
    a.inv255 = 1.f / 255.f;
    for (int c = 0; c < 3; ++c) {
        a.mean[c] = h_mean[c];
        a.istd[c] = 1.f / h_std[c];
    }
    a.out32 = out32;
    a.out16 = out16;
    const int npix = oh * ow;
    const int bx = std::min((npix + 255) / 256, 1024);
    dim3 grid(bx, static_cast<unsigned>(s->n));
    resize_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}
}  // namespace
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

scn_status scn_thumbs(scn_seq* s, uint8_t* d_thumb, void* stream) {
    if (!s || !d_thumb) return SCN_EINVAL;
    const int W = s->table->W, H = s->table->H;
    if (W % 64 || H % 36 || W / 64 != H / 36) return SCN_EUNSUPPORTED;
    if (s->n == 0) return SCN_OK;
    if (s->n > 0x7fffffff) return SCN_ERANGE;
    scn::thumbs_kernel<<<static_cast<unsigned>(s->n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        s->table->d_nv12, s->table->frame_stride, W, W / 64, s->d_slot, d_thumb);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // extern "C"
