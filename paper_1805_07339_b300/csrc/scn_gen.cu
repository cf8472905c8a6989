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
    // the same when |d| <= W: at most one wrap, no loop (selects only)
    __device__ __forceinline__ void step1(int d, int W) {
        r += d;
        const bool up = r >= W, down = r < 0;
        r += up ? -W : (down ? W : 0);
        q += up ? 1 : (down ? -1 : 0);
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

// One 16-byte vector (16 luma samples of one row, or 8 U/V pairs of one chroma
// row) of frame f, shot fields sh.  Along a row the sample index q steps by 1, so
// the counter s_pix + (2q+1) kGolden steps by 2 kGolden, and floor(gx (x - dt) / W)
// is kept as quotient and remainder.
__device__ __forceinline__ uint4 gen_vector(const GenArgs& a, int64_t f, const scn_shot& sh, int row, int vec) {
    const int dt = static_cast<int>(f - sh.start);
    uint8_t b[16];
    if (row < a.H) {
        const int y = row;
        const int x0 = vec * 16;
        const int base = sh.base[0] + floordiv_pos(sh.gy[0] * y, a.H);
        const uint64_t q0 = (static_cast<uint64_t>(f) * 3 * a.H + y) * a.W + x0;
        uint64_t c = a.s_pix + (2 * q0 + 1) * kGolden;
        FloorStep rx;
        rx.init(sh.gx[0] * (x0 - dt), a.W);
        const int gx = sh.gx[0];
        if (abs(gx) <= a.W) {  // every frame of 32 columns or more (|gx| <= 32)
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int v = base + rx.q + noise_from_counter(c);
                b[i] = static_cast<uint8_t>(min(max(v, 16), 235));
                c += 2 * kGolden;
                rx.step1(gx, a.W);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int v = base + rx.q + noise_from_counter(c);
                b[i] = static_cast<uint8_t>(min(max(v, 16), 235));
                c += 2 * kGolden;
                rx.step(gx, a.W);
            }
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
            rx[pl - 1].init(sh.gx[pl] * (2 * cx0 - dt), a.W);
            base[pl - 1] = sh.base[pl] + floordiv_pos(sh.gy[pl] * (2 * cy), a.H);
            gx2[pl - 1] = 2 * sh.gx[pl];
        }
        if (abs(gx2[0]) <= a.W && abs(gx2[1]) <= a.W) {  // every frame of 64 columns or more
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int pl = 0; pl < 2; ++pl) {
                    const int v = base[pl] + rx[pl].q + noise_from_counter(c[pl]);
                    b[2 * j + pl] = static_cast<uint8_t>(min(max(v, 16), 240));
                    c[pl] += 2 * kGolden;
                    rx[pl].step1(gx2[pl], a.W);
                }
            }
        } else {
#pragma unroll
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
    }
    uint4 o;
    o.x = b[0] | (b[1] << 8) | (b[2] << 16) | (static_cast<unsigned>(b[3]) << 24);
    o.y = b[4] | (b[5] << 8) | (b[6] << 16) | (static_cast<unsigned>(b[7]) << 24);
    o.z = b[8] | (b[9] << 8) | (b[10] << 16) | (static_cast<unsigned>(b[11]) << 24);
    o.w = b[12] | (b[13] << 8) | (b[14] << 16) | (static_cast<unsigned>(b[15]) << 24);
    return o;
}

constexpr int kGenThreads = 256;
constexpr int kGenVecsPerThread = 4;  // vectors of one frame per thread (about)

// blockIdx.y walks the frames, blockIdx.x spans one frame's vectors: the frame's
// shot is found once per block (one thread) and read from shared memory, and the
// vector index within a frame stays in 32 bits (rows x W/16 < 2^31, checked on the host).
__global__ void __launch_bounds__(kGenThreads) gen_kernel(GenArgs a) {
    __shared__ scn_shot s_shot;
    const int vecs = a.W / 16;
    const int per_frame = (a.H + a.H / 2) * vecs;
    for (int64_t k = blockIdx.y; k < a.count; k += gridDim.y) {
        const int64_t f = a.frames ? a.frames[k] : a.first + k;
        __syncthreads();  // the previous frame's readers are done with s_shot
        if (threadIdx.x == 0) s_shot = *shot_of(a.shots, a.nshots, f);
        __syncthreads();
        const scn_shot sh = s_shot;
        uint8_t* out = a.out + k * a.stride;
        for (int r = blockIdx.x * kGenThreads + threadIdx.x; r < per_frame; r += gridDim.x * kGenThreads) {
            const int row = r / vecs;
            const int vec = r - row * vecs;
            *reinterpret_cast<uint4*>(out + static_cast<int64_t>(row) * a.W + vec * 16) = gen_vector(a, f, sh, row, vec);
        }
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
    const int64_t per_frame = (static_cast<int64_t>(a.H) + a.H / 2) * (a.W / 16);
    if (per_frame > 0x7fffffff) return SCN_ERANGE;
    const int64_t bx = (per_frame + kGenThreads * kGenVecsPerThread - 1) / (kGenThreads * kGenVecsPerThread);
    const dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(std::min<int64_t>(count, 65535)));
    gen_kernel<<<grid, kGenThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
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
