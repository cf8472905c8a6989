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

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// SplitMix64 finaliser of a counter value c = s + (i+1) * kGolden
__device__ __forceinline__ uint64_t sm_mix(uint64_t v) {
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    return v ^ (v >> 31);
}

// noise of the sample whose first counter value is c (= s_pix + (2q+1) kGolden; the
// second draw's counter is c + kGolden)
__device__ __forceinline__ int noise_from_counter(uint64_t c) {
    const uint64_t w0 = sm_mix(c);
    const uint64_t w1 = sm_mix(c + kGolden);
    unsigned sum = __dp4a(static_cast<unsigned>(w0), 0x01010101u, 0u);
    sum = __dp4a(static_cast<unsigned>(w0 >> 32), 0x01010101u, sum);
    sum = __dp4a(static_cast<unsigned>(w1), 0x01010101u, sum);
    return (static_cast<int>(sum) - 1514) >> 5;  // arithmetic shift = floor division by 32
}

// floor(n / W) kept as quotient and remainder while n steps by d (W > 0)
struct FloorStep {
    int q, r;
    __device__ __forceinline__ void init(int n, int W) {
        q = n / W;
        r = n - q * W;
        if (r < 0) {
            r += W;
            --q;
        }
    }
    __device__ __forceinline__ void step(int d, int W) {
        r += d;
        while (r >= W) {
            r -= W;
            ++q;
        }
        while (r < 0) {
            r += W;
            --q;
        }
    }
};

__device__ __forceinline__ int floordiv_pos(int a, int b) {
    // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
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
        // Along a row the sample index q steps by 1, so the counter s_pix + (2q+1) kGolden
        // steps by 2 kGolden, and floor(gx (x - dt) / W) is kept as quotient and remainder.
        if (row < a.H) {
            const int y = row;
            const int x0 = vec * 16;
            const int base = sh->base[0] + floordiv_pos(sh->gy[0] * y, a.H);
            const uint64_t q0 = (static_cast<uint64_t>(f) * 3 * a.H + y) * a.W + x0;
            uint64_t c = a.s_pix + (2 * q0 + 1) * kGolden;
            FloorStep rx;
            rx.init(sh->gx[0] * (x0 - dt), a.W);
            const int gx = sh->gx[0];
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int v = base + rx.q + noise_from_counter(c);
                b[i] = static_cast<uint8_t>(min(max(v, 16), 235));
                c += 2 * kGolden;
                rx.step(gx, a.W);
            }
        } else {
            const int cy = row - a.H;
            const int Wc = a.W / 2, Hc = a.H / 2;
            const int cx0 = vec * 8;
            uint64_t c[2];
            FloorStep rx[2];
            int base[2], gx2[2];
#pragma unroll
            for (int pl = 1; pl <= 2; ++pl) {
                const uint64_t q0 = ((static_cast<uint64_t>(f) * 3 + pl) * Hc + cy) * Wc + cx0;
                c[pl - 1] = a.s_pix + (2 * q0 + 1) * kGolden;
                rx[pl - 1].init(sh->gx[pl] * (2 * cx0 - dt), a.W);
                base[pl - 1] = sh->base[pl] + floordiv_pos(sh->gy[pl] * (2 * cy), a.H);
                gx2[pl - 1] = 2 * sh->gx[pl];
            }
#pragma unroll 2
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int pl = 0; pl < 2; ++pl) {
                    const int v = base[pl] + rx[pl].q + noise_from_counter(c[pl]);
                    b[2 * j + pl] = static_cast<uint8_t>(min(max(v, 16), 240));
                    c[pl] += 2 * kGolden;
                    rx[pl].step(gx2[pl], a.W);
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
