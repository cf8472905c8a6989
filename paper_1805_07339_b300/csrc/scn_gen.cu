// Synthetic NV12 video generator on the GPU (stands in for decoded frames).
//
// Definition (shared with the CPU oracle only as a specification, not as code):
//   value(plane p, luma coords x,y, frame f) = base_p + floor(gx_p (x - dt) / W)
//       + floor(gy_p y / H) + noise(q), clamped to [16,235] (Y) or [16,240] (U,V),
//   dt = f - shot start, q = ((f*3 + p) * H_p + y_p) * W_p + x_p in plane coords,
//   noise(q) = floor((S - 1514) / 32), S = the 8 bytes of SM(s_pix, 2q) plus the
//   low 4 bytes of SM(s_pix, 2q+1): Irwin-Hall with 12 uniform bytes, sigma 8.
// SplitMix64 counter form: SM(s, i) = finalise(s + (i+1) * 0x9E3779B97F4A7C15).
#include <cuda_runtime.h>

#include "scn_internal.h"

namespace scn {
namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t s, uint64_t i) {
    uint64_t v = s + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    return v ^ (v >> 31);
}

__device__ __forceinline__ int floordiv_pos(int a, int b) {
    // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ int noise_at(uint64_t s_pix, uint64_t q) {
    const uint64_t w0 = sm64(s_pix, 2 * q);
    const uint64_t w1 = sm64(s_pix, 2 * q + 1);
    unsigned sum = __dp4a(static_cast<unsigned>(w0), 0x01010101u, 0u);
    sum = __dp4a(static_cast<unsigned>(w0 >> 32), 0x01010101u, sum);
    sum = __dp4a(static_cast<unsigned>(w1), 0x01010101u, sum);
    return (static_cast<int>(sum) - 1514) >> 5;  // arithmetic shift = floor division by 32
}

struct GenArgs {
    const scn_shot* shots;
    int nshots;
    int W, H;
    uint64_t s_pix;
    const int64_t* frames;  // null: frame = first + k
    int64_t first;
    int64_t count;
    int64_t stride;
    uint8_t* out;
};

__device__ __forceinline__ const scn_shot* shot_of(const scn_shot* shots, int nshots, int64_t f) {
    int lo = 0, hi = nshots - 1;  // last shot with start <= f
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (shots[mid].start <= f) lo = mid; else hi = mid - 1;
    }
    return shots + lo;
}

__global__ void __launch_bounds__(256) gen_kernel(GenArgs a) {
    const int vecs = a.W / 16;
    const int rows = a.H + a.H / 2;
    const int64_t per_frame = static_cast<int64_t>(rows) * vecs;
    const int64_t total = per_frame * a.count;
    for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < total;
         w += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = w / per_frame;
        const int64_t r = w - k * per_frame;
        const int row = static_cast<int>(r / vecs);
        const int vec = static_cast<int>(r - static_cast<int64_t>(row) * vecs);
        const int64_t f = a.frames ? a.frames[k] : a.first + k;
        const scn_shot* sh = shot_of(a.shots, a.nshots, f);
        const int dt = static_cast<int>(f - sh->start);
        uint8_t b[16];
        if (row < a.H) {
            const int y = row;
            const int ramp_y = floordiv_pos(sh->gy[0] * y, a.H);
            const uint64_t qrow = (static_cast<uint64_t>(f) * 3 * a.H + y) * a.W;
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int x = vec * 16 + i;
                int v = sh->base[0] + floordiv_pos(sh->gx[0] * (x - dt), a.W) + ramp_y +
                        noise_at(a.s_pix, qrow + x);
                b[i] = static_cast<uint8_t>(min(max(v, 16), 235));
            }
        } else {
            const int cy = row - a.H;
            const int Wc = a.W / 2, Hc = a.H / 2;
#pragma unroll 2
            for (int j = 0; j < 8; ++j) {
                const int cx = vec * 8 + j;
#pragma unroll
                for (int pl = 1; pl <= 2; ++pl) {
                    const uint64_t q = ((static_cast<uint64_t>(f) * 3 + pl) * Hc + cy) * Wc + cx;
                    int v = sh->base[pl] + floordiv_pos(sh->gx[pl] * (2 * cx - dt), a.W) +
                            floordiv_pos(sh->gy[pl] * (2 * cy), a.H) + noise_at(a.s_pix, q);
                    b[2 * j + pl - 1] = static_cast<uint8_t>(min(max(v, 16), 240));
                }
            }
        }
        uint4 o;
        o.x = b[0] | (b[1] << 8) | (b[2] << 16) | (static_cast<unsigned>(b[3]) << 24);
        o.y = b[4] | (b[5] << 8) | (b[6] << 16) | (static_cast<unsigned>(b[7]) << 24);
        o.z = b[8] | (b[9] << 8) | (b[10] << 16) | (static_cast<unsigned>(b[11]) << 24);
        o.w = b[12] | (b[13] << 8) | (b[14] << 16) | (static_cast<unsigned>(b[15]) << 24);
        *reinterpret_cast<uint4*>(a.out + k * a.stride + static_cast<int64_t>(row) * a.W + vec * 16) = o;
    }
}

uint64_t host_sm64(uint64_t s, uint64_t i) {
    uint64_t v = s + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    return v ^ (v >> 31);
}

scn_status launch_gen(const scn_video* v, const int64_t* d_frames, int64_t first, int64_t count, uint8_t* d_out,
                      int64_t stride, void* stream) {
    if (!v || !d_out || count < 0) return SCN_EINVAL;
    const int64_t fb = static_cast<int64_t>(v->p.width) * v->p.height * 3 / 2;
    if (stride < fb || (stride % 16) || !aligned16(d_out)) return SCN_EINVAL;
    if (!d_frames && (first < 0 || first + count > v->p.num_frames)) return SCN_ERANGE;
    if (count == 0) return SCN_OK;
    GenArgs a;
    a.shots = v->d_shots;
    a.nshots = static_cast<int>(v->shots.size());
    a.W = v->p.width;
    a.H = v->p.height;
    a.s_pix = host_sm64(host_sm64(v->p.master_seed, v->p.video_id), 2);
    a.frames = d_frames;
    a.first = first;
    a.count = count;
    a.stride = stride;
    a.out = d_out;
    const int sms = device_sm_count();
    if (sms <= 0) return SCN_EUNSUPPORTED;
    const int64_t work = (static_cast<int64_t>(a.H) * 3 / 2) * (a.W / 16) * count;
    const int64_t blocks = std::min<int64_t>((work + 255) / 256, static_cast<int64_t>(sms) * 16);
    gen_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // namespace
}  // namespace scn

extern "C" {

scn_status scn_generate(const scn_video* v, uint8_t* d_out, int64_t first_frame, int64_t count,
                        int64_t frame_stride, void* stream) {
    return scn::launch_gen(v, nullptr, first_frame, count, d_out, frame_stride, stream);
}

scn_status scn_generate_frames(const scn_video* v, const int64_t* d_frames, int64_t n, uint8_t* d_out,
                               int64_t frame_stride, void* stream) {
    if (n > 0 && !d_frames) return SCN_EINVAL;
    return scn::launch_gen(v, d_frames, 0, n, d_out, frame_stride, stream);
}

}  // extern "C"
