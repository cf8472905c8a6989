// The learned boundary proposal: a tiny BF16 CNN over pairs of 36x64 luma
// thumbnails, forward and training on the GPU.
//
// Network (fp32 master weights; BF16 weights and activations, FP32 accumulation):
//   x  = [(Y_prev - 128)/64, (Y_cur - 128)/64]                 2 x 36 x 64
//   a1 = relu(conv3x3 s2 p1, 2 -> 16)                          16 x 18 x 32
//   a2 = relu(conv3x3 s2 p1, 16 -> 32)                         32 x 9 x 16
//   a3 = relu(conv3x3 s2 p1, 32 -> 32)                         32 x 5 x 8
//   g = mean(a3), h = relu(F1 g + c1) (64), z = F2 h + c2      logit
// Loss: BCE with logits, positive weight w; optimiser Adam.
//
// Kernels:
//  * conv forward: implicit GEMM on tcgen05 - the 128 x K im2col tile of 128
//    output positions (any pairs) and the COUT x K weight tile in shared
//    memory (core-matrix layout), K/16 MMAs into a TMEM accumulator, bias +
//    ReLU + BF16 in the epilogue.  Activations are NHWC.
//  * conv backward-data (layers 2, 3): tcgen05 GEMM dXcol = dU * W (M = 128
//    rows, N = K columns, contraction over COUT), then a gather col2im that
//    applies the ReLU mask of the layer below.
//  * conv backward-weights, head forward/backward, Adam: CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "scn_internal.h"
#include "scn_ptx.cuh"
#include "scn_tc.cuh"

namespace scn {
namespace cnn {

// ---------------------------------------------------------------------------
// geometry and parameter layout (flat fp32, the oracle's order)
// ---------------------------------------------------------------------------
template <int L>
struct Geo;
template <>
struct Geo<1> {
    static constexpr int CIN = 2, COUT = 16, HIN = 36, WIN = 64;
};
template <>
struct Geo<2> {
    static constexpr int CIN = 16, COUT = 32, HIN = 18, WIN = 32;
};
template <>
struct Geo<3> {
    static constexpr int CIN = 32, COUT = 32, HIN = 9, WIN = 16;
};
template <int L>
struct Shape : Geo<L> {
    using G = Geo<L>;
    static constexpr int HO = (G::HIN - 1) / 2 + 1, WO = (G::WIN - 1) / 2 + 1, P = HO * WO;
    static constexpr int K = G::CIN * 9, KP = (K + 15) / 16 * 16;
};

// offsets into the flat parameter vector
constexpr int kW1 = 0, kB1 = kW1 + 16 * 2 * 9, kW2 = kB1 + 16, kB2 = kW2 + 32 * 16 * 9, kW3 = kB2 + 32,
              kB3 = kW3 + 32 * 32 * 9, kF1 = kB3 + 32, kC1 = kF1 + 64 * 32, kF2 = kC1 + 64, kC2 = kF2 + 64,
              kNParams = kC2 + 1;
static_assert(kNParams == 16369, "parameter count");

constexpr uint64_t kWaitNs = 2000000000ull;

struct Net {
    // parameters (device)
    float* master;          // [kNParams]
    float* adam_m;
    float* adam_v;
    float* grad;            // [kNParams]
    __nv_bfloat16* w1b;     // [16][32]   (k = tap*2 + ci, zero padded)
    __nv_bfloat16* w2b;     // [32][144]  (k = tap*16 + ci)
    __nv_bfloat16* w3b;     // [32][288]
    __nv_bfloat16* w2t;     // [144][32]  transposed (backward-data)
    __nv_bfloat16* w3t;     // [288][32]
    __nv_bfloat16* f1b;     // [64][32]
    __nv_bfloat16* f2b;     // [64]
    // activations of the last batch (device)
    __nv_bfloat16 *a1, *a2, *a3;   // NHWC
    float *g, *v, *z;              // head
    __nv_bfloat16 *du1, *du2, *du3;
    float *dx2, *dx3;              // im2col-shaped data gradients
    float* loss;
    int* status;
    int64_t max_batch;
    int64_t step;
    void* block;
};

// ---------------------------------------------------------------------------
// conv forward on tcgen05
// ---------------------------------------------------------------------------
struct ConvFwdArgs {
    const uint8_t* thumbs;    // layer 1: uint8 [frames][36][64]
    const int32_t* prev;      // layer 1: thumbnail index of each pair's first frame (null: pair b = (b, b+1))
    const int32_t* cur;
    const __nv_bfloat16* x;   // layers 2, 3: NHWC input [pairs][HIN*WIN][CIN]
    const __nv_bfloat16* w;   // [COUT][KP]
    const float* bias;        // [COUT]
    __nv_bfloat16* y;         // NHWC output [pairs][P][COUT]
    int64_t pairs;
    int* status;
};

template <int L>
struct ConvSmem {
    using S = Shape<L>;
    static constexpr int A_BYTES = 128 * S::KP * 2, B_BYTES = S::COUT * S::KP * 2;
    static constexpr int BYTES = A_BYTES + B_BYTES + 64;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return static_cast<uint32_t>(__bfloat16_as_ushort(a)) | (static_cast<uint32_t>(__bfloat16_as_ushort(b)) << 16);
}

// 8 consecutive im2col values (columns 8j..8j+7) of output row (pair b, position pos)
template <int L>
__device__ __forceinline__ uint4 im2col_chunk(const ConvFwdArgs& a, int64_t b, int pos, int j) {
    using S = Shape<L>;
    const int oy = pos / S::WO, ox = pos - (pos / S::WO) * S::WO;
    if constexpr (L == 1) {
        // k = tap*2 + channel: taps 4j .. 4j+3, channel 0 = previous thumbnail, 1 = current
        const int ip = a.prev ? a.prev[b] : static_cast<int>(b);
        const int ic = a.cur ? a.cur[b] : static_cast<int>(b + 1);
        const uint8_t* tp = a.thumbs + static_cast<int64_t>(ip) * 2304;
        const uint8_t* tcur = a.thumbs + static_cast<int64_t>(ic) * 2304;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int tap = 4 * j + q;
            float v0 = 0.f, v1 = 0.f;
            if (tap < 9) {
                const int iy = 2 * oy - 1 + tap / 3, ix = 2 * ox - 1 + tap % 3;
                if (iy >= 0 && iy < S::HIN && ix >= 0 && ix < S::WIN) {
                    v0 = (static_cast<float>(__ldg(tp + iy * 64 + ix)) - 128.f) * (1.f / 64.f);
                    v1 = (static_cast<float>(__ldg(tcur + iy * 64 + ix)) - 128.f) * (1.f / 64.f);
                }
            }
            w[q] = pack_bf16(v0, v1);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    } else {
        // k = tap*CIN + channel: 8 channels of one tap
        const int tap = (8 * j) / S::CIN, c0 = (8 * j) % S::CIN;
        const int iy = 2 * oy - 1 + tap / 3, ix = 2 * ox - 1 + tap % 3;
        if (tap >= 9 || iy < 0 || iy >= S::HIN || ix < 0 || ix >= S::WIN) return make_uint4(0, 0, 0, 0);
        const __nv_bfloat16* p = a.x + ((b * S::HIN + iy) * S::WIN + ix) * S::CIN + c0;
        return __ldg(reinterpret_cast<const uint4*>(p));
    }
}

template <int L>
__global__ void __launch_bounds__(128) conv_fwd_tc(const __grid_constant__ ConvFwdArgs a) {
    using S = Shape<L>;
    using M = ConvSmem<L>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* As = smem;
    uint8_t* Bs = smem + M::A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + M::A_BYTES + M::B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights -> B tile (core layout), once
    for (int e = tid; e < S::COUT * (S::KP / 8); e += 128) {
        const int n = e / (S::KP / 8), j = e % (S::KP / 8);
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.w + n * S::KP + 8 * j));
        *reinterpret_cast<uint4*>(Bs + tc::core_offset(n, 8 * j, S::KP)) = v;
    }
    if (tid == 0) {
        ptx::mbar_init(mbar, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 32);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t a_addr = ptx::smem_u32(As), b_addr = ptx::smem_u32(Bs);
    constexpr uint32_t kSbo = (S::KP / 8) * 128;
    constexpr uint32_t idesc = tc::idesc_bf16(128, S::COUT);
    const int64_t rows = a.pairs * S::P;
    const int64_t tiles = (rows + 127) / 128;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // A tile: row tid of this tile
        const int64_t r = t * 128 + tid;
        const bool live = r < rows;
        const int64_t b = live ? r / S::P : 0;
        const int pos = live ? static_cast<int>(r - b * S::P) : 0;
#pragma unroll 4
        for (int j = 0; j < S::KP / 8; ++j) {
            const uint4 v = live ? im2col_chunk<L>(a, b, pos, j) : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(As + tc::core_offset(tid, 8 * j, S::KP)) = v;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < S::KP / 16; ++kk) {
                tc::mma(tmem, tc::smem_desc(a_addr + kk * 256, 128, kSbo), tc::smem_desc(b_addr + kk * 256, 128, kSbo),
                        idesc, kk > 0 ? 1u : 0u);
            }
            tc::commit(mbar);
        }
        if (ok && !ptx::mbar_wait_bounded(mbar, phase, kWaitNs)) {
            ok = false;
            atomicOr(a.status, kStatusTimeout);
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // epilogue: thread = row, COUT columns
        uint32_t acc[S::COUT];
#pragma unroll
        for (int c0 = 0; c0 < S::COUT; c0 += 16) {
            uint32_t q[16];
            tc::ld16(tmem + ((32u * warp) << 16) + c0, q);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[c0 + i] = q[i];
        }
        tc::wait_ld();
        if (live && ok) {
            uint32_t out[S::COUT / 2];
#pragma unroll
            for (int c = 0; c < S::COUT; c += 2) {
                const float v0 = fmaxf(__uint_as_float(acc[c]) + __ldg(a.bias + c), 0.f);
                const float v1 = fmaxf(__uint_as_float(acc[c + 1]) + __ldg(a.bias + c + 1), 0.f);
                out[c / 2] = pack_bf16(v0, v1);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.y + r * S::COUT);
#pragma unroll
            for (int q = 0; q < S::COUT / 8; ++q) dst[q] = make_uint4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------------------------------
// head forward: warp per pair
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) head_fwd(const __nv_bfloat16* __restrict__ a3, const __nv_bfloat16* f1b,
                                                const float* c1, const __nv_bfloat16* f2b, const float* c2, float* g_out,
                                                float* v_out, float* z, int64_t pairs) {
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    if (b >= pairs) return;
    float s = 0.f;
    const __nv_bfloat16* p = a3 + b * 40 * 32 + lane;
    for (int pos = 0; pos < 40; ++pos) s += __bfloat162float(p[pos * 32]);
    const float g = s * (1.f / 40.f);
    float v0 = c1[lane], v1 = c1[lane + 32];
    for (int c = 0; c < 32; ++c) {
        const float gc = __shfl_sync(0xffffffffu, g, c);
        v0 = fmaf(__bfloat162float(f1b[lane * 32 + c]), gc, v0);
        v1 = fmaf(__bfloat162float(f1b[(lane + 32) * 32 + c]), gc, v1);
    }
    float zz = __bfloat162float(f2b[lane]) * fmaxf(v0, 0.f) + __bfloat162float(f2b[lane + 32]) * fmaxf(v1, 0.f);
    for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
    if (g_out) {
        g_out[b * 32 + lane] = g;
        v_out[b * 64 + lane] = v0;
        v_out[b * 64 + 32 + lane] = v1;
    }
    if (lane == 0) z[b] = zz + c2[0];
}

// ---------------------------------------------------------------------------
// fp32 master -> BF16 operand layouts
// ---------------------------------------------------------------------------
__global__ void prep_weights(const float* m, __nv_bfloat16* w1b, __nv_bfloat16* w2b, __nv_bfloat16* w3b,
                             __nv_bfloat16* w2t, __nv_bfloat16* w3t, __nv_bfloat16* f1b, __nv_bfloat16* f2b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // conv weights W[co][ci][di][dj] -> [co][tap*CIN + ci]
    if (i < 16 * 32) {
        const int co = i / 32, k = i % 32;
        float v = 0.f;
        if (k < 18) v = m[kW1 + (co * 2 + k % 2) * 9 + k / 2];
        w1b[i] = __float2bfloat16_rn(v);
    }
    if (i < 32 * 144) {
        const int co = i / 144, k = i % 144, tap = k / 16, ci = k % 16;
        const __nv_bfloat16 v = __float2bfloat16_rn(m[kW2 + (co * 16 + ci) * 9 + tap]);
        w2b[i] = v;
        w2t[k * 32 + co] = v;
    }
    if (i < 32 * 288) {
        const int co = i / 288, k = i % 288, tap = k / 32, ci = k % 32;
        const __nv_bfloat16 v = __float2bfloat16_rn(m[kW3 + (co * 32 + ci) * 9 + tap]);
        w3b[i] = v;
        w3t[k * 32 + co] = v;
    }
    if (i < 64 * 32) f1b[i] = __float2bfloat16_rn(m[kF1 + i]);
    if (i < 64) f2b[i] = __float2bfloat16_rn(m[kF2 + i]);
}

template <int L>
scn_status launch_conv_fwd(const ConvFwdArgs& a, cudaStream_t st) {
    static int attr_dev = -1;
    int dev = 0;
    SCN_CUDA_TRY(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_fwd_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          ConvSmem<L>::BYTES));
        attr_dev = dev;
    }
    const int64_t tiles = (a.pairs * Shape<L>::P + 127) / 128;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(sms) * 4));
    conv_fwd_tc<L><<<grid, 128, ConvSmem<L>::BYTES, st>>>(a);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

// forward of one chunk of at most max_batch pairs; keeps head intermediates when train is set
scn_status forward_chunk(Net* n, const uint8_t* thumbs, const int32_t* prev, const int32_t* cur, int64_t pairs,
                         float* logits, bool train, cudaStream_t st) {
    ConvFwdArgs a{};
    a.thumbs = thumbs;
    a.prev = prev;
    a.cur = cur;
    a.pairs = pairs;
    a.status = n->status;
    a.w = n->w1b;
    a.bias = n->master + kB1;
    a.y = n->a1;
    scn_status s = launch_conv_fwd<1>(a, st);
    if (s != SCN_OK) return s;
    a.x = n->a1;
    a.w = n->w2b;
    a.bias = n->master + kB2;
    a.y = n->a2;
    s = launch_conv_fwd<2>(a, st);
    if (s != SCN_OK) return s;
    a.x = n->a2;
    a.w = n->w3b;
    a.bias = n->master + kB3;
    a.y = n->a3;
    s = launch_conv_fwd<3>(a, st);
    if (s != SCN_OK) return s;
    const int64_t blocks = (pairs + 7) / 8;
    head_fwd<<<static_cast<unsigned>(blocks), 256, 0, st>>>(n->a3, n->f1b, n->master + kC1, n->f2b, n->master + kC2,
                                                            train ? n->g : nullptr, train ? n->v : nullptr, logits,
                                                            pairs);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

// ---------------------------------------------------------------------------
// training: head backward (warp per pair, register accumulation per warp)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) head_bwd(const float* __restrict__ z, const float* __restrict__ y,
                                                const float* __restrict__ g, const float* __restrict__ v,
                                                const __nv_bfloat16* __restrict__ a3, const __nv_bfloat16* f1b,
                                                const __nv_bfloat16* f2b, float pos_weight, int64_t pairs,
                                                float* grad, __nv_bfloat16* du3, float* loss) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    float dF1a[32], dF1b[32];  // rows j = lane and lane + 32
#pragma unroll
    for (int c = 0; c < 32; ++c) dF1a[c] = dF1b[c] = 0.f;
    float dc1a = 0.f, dc1b = 0.f, dF2a = 0.f, dF2b = 0.f, dc2 = 0.f, lsum = 0.f;
    const float inv_b = 1.f / static_cast<float>(pairs);
    for (int64_t b = w0; b < pairs; b += nw) {
        const float zz = z[b], yy = y[b];
        const float sig = 1.f / (1.f + __expf(-zz));
        const float dz = (pos_weight * yy * (sig - 1.f) + (1.f - yy) * sig) * inv_b;
        // softplus(-z), softplus(z) for the loss
        const float spn = fmaxf(-zz, 0.f) + log1pf(__expf(-fabsf(zz)));
        const float spp = fmaxf(zz, 0.f) + log1pf(__expf(-fabsf(zz)));
        lsum += (pos_weight * yy * spn + (1.f - yy) * spp) * inv_b;
        const float va = v[b * 64 + lane], vb = v[b * 64 + 32 + lane];
        const float ha = fmaxf(va, 0.f), hb = fmaxf(vb, 0.f);
        dF2a += dz * ha;
        dF2b += dz * hb;
        dc2 += dz;
        const float dva = va > 0.f ? dz * __bfloat162float(f2b[lane]) : 0.f;
        const float dvb = vb > 0.f ? dz * __bfloat162float(f2b[lane + 32]) : 0.f;
        dc1a += dva;
        dc1b += dvb;
        const float gl = g[b * 32 + lane];
        float dg = 0.f;  // for channel c = lane
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float gc = __shfl_sync(0xffffffffu, gl, c);
            dF1a[c] = fmaf(dva, gc, dF1a[c]);
            dF1b[c] = fmaf(dvb, gc, dF1b[c]);
        }
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const float dvj_a = __shfl_sync(0xffffffffu, dva, j), dvj_b = __shfl_sync(0xffffffffu, dvb, j);
            dg = fmaf(__bfloat162float(f1b[j * 32 + lane]), dvj_a, dg);
            dg = fmaf(__bfloat162float(f1b[(j + 32) * 32 + lane]), dvj_b, dg);
        }
        const float da3 = dg * (1.f / 40.f);
        const __nv_bfloat16* ap = a3 + b * 40 * 32 + lane;
        __nv_bfloat16* dp = du3 + b * 40 * 32 + lane;
        for (int pos = 0; pos < 40; ++pos)
            dp[pos * 32] = __float2bfloat16_rn(__bfloat162float(ap[pos * 32]) > 0.f ? da3 : 0.f);
    }
    if (w0 >= pairs) return;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        atomicAdd(grad + kF1 + lane * 32 + c, dF1a[c]);
        atomicAdd(grad + kF1 + (lane + 32) * 32 + c, dF1b[c]);
    }
    atomicAdd(grad + kC1 + lane, dc1a);
    atomicAdd(grad + kC1 + lane + 32, dc1b);
    atomicAdd(grad + kF2 + lane, dF2a);
    atomicAdd(grad + kF2 + lane + 32, dF2b);
    // dc2 and the loss are the same in every lane (they depend on z only)
    if (lane == 0) {
        atomicAdd(grad + kC2, dc2);
        atomicAdd(loss, lsum);
    }
}

// ---------------------------------------------------------------------------
// conv backward-data on tcgen05: dXcol[r][k] = sum_co dU[r][co] * W[co][k]
// (M = 128 rows, N = KP columns in halves of at most 144, contraction COUT)
// ---------------------------------------------------------------------------
struct ConvBwdArgs {
    const __nv_bfloat16* du;   // [rows][COUT]
    const __nv_bfloat16* wt;   // [KP][COUT]
    float* dxcol;              // [rows][KP]
    int64_t pairs;
    int* status;
};

template <int L>
struct BwdSmem {
    using S = Shape<L>;
    static constexpr int A_BYTES = 128 * S::COUT * 2, B_BYTES = S::KP * S::COUT * 2;
    static constexpr int BYTES = A_BYTES + B_BYTES + 64;
};

template <int L>
__global__ void __launch_bounds__(128) conv_bwd_data_tc(const __grid_constant__ ConvBwdArgs a) {
    using S = Shape<L>;
    using M = BwdSmem<L>;
    constexpr int NH = S::KP > 144 ? 2 : 1;   // N halves
    constexpr int NN = S::KP / NH;            // 144 for both layers
    static_assert(NN % 16 == 0 && NN <= 256, "N");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* As = smem;
    uint8_t* Bs = smem + M::A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + M::A_BYTES + M::B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < S::KP * (S::COUT / 8); e += 128) {
        const int n = e / (S::COUT / 8), j = e % (S::COUT / 8);
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.wt + n * S::COUT + 8 * j));
        *reinterpret_cast<uint4*>(Bs + tc::core_offset(n, 8 * j, S::COUT)) = v;
    }
    if (tid == 0) {
        ptx::mbar_init(mbar, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t a_addr = ptx::smem_u32(As), b_addr = ptx::smem_u32(Bs);
    constexpr uint32_t kSbo = (S::COUT / 8) * 128;
    constexpr uint32_t idesc = tc::idesc_bf16(128, NN);
    const int64_t rows = a.pairs * S::P;
    const int64_t tiles = (rows + 127) / 128;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t r = t * 128 + tid;
        const bool live = r < rows;
#pragma unroll
        for (int j = 0; j < S::COUT / 8; ++j) {
            const uint4 v = live ? __ldg(reinterpret_cast<const uint4*>(a.du + r * S::COUT + 8 * j)) : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(As + tc::core_offset(tid, 8 * j, S::COUT)) = v;
        }
        tc::fence_proxy_async();
        for (int h = 0; h < NH; ++h) {
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t bh = b_addr + (h * NN / 8) * kSbo;
#pragma unroll
                for (int kk = 0; kk < S::COUT / 16; ++kk)
                    tc::mma(tmem, tc::smem_desc(a_addr + kk * 256, 128, kSbo), tc::smem_desc(bh + kk * 256, 128, kSbo),
                            idesc, kk > 0 ? 1u : 0u);
                tc::commit(mbar);
            }
            if (ok && !ptx::mbar_wait_bounded(mbar, phase, kWaitNs)) {
                ok = false;
                atomicOr(a.status, kStatusTimeout);
            }
            phase ^= 1u;
            tc::fence_after_sync();
            float* dst = a.dxcol + r * S::KP + h * NN;
#pragma unroll 1
            for (int c0 = 0; c0 < NN; c0 += 16) {
                uint32_t q[16];
                tc::ld16(tmem + ((32u * warp) << 16) + c0, q);
                tc::wait_ld();
                if (live && ok) {
                    float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        d4[i] = make_float4(__uint_as_float(q[4 * i]), __uint_as_float(q[4 * i + 1]),
                                            __uint_as_float(q[4 * i + 2]), __uint_as_float(q[4 * i + 3]));
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// col2im of layer L's data gradient into its input positions, times the ReLU
// mask of that input (the previous layer's activation); BF16 out.
template <int L>
__global__ void col2im_mask(const float* __restrict__ dxcol, const __nv_bfloat16* __restrict__ act,
                            __nv_bfloat16* __restrict__ du_prev, int64_t pairs) {
    using S = Shape<L>;
    const int64_t total = pairs * S::HIN * S::WIN * S::CIN;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int ci = static_cast<int>(i % S::CIN);
        const int64_t q = i / S::CIN;
        const int ix = static_cast<int>(q % S::WIN);
        const int iy = static_cast<int>((q / S::WIN) % S::HIN);
        const int64_t b = q / (S::WIN * S::HIN);
        float s = 0.f;
        // output (oy, ox) with tap (di, dj): iy = 2 oy - 1 + di, ix = 2 ox - 1 + dj
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            const int ty = iy + 1 - di;
            if (ty < 0 || (ty & 1)) continue;
            const int oy = ty >> 1;
            if (oy >= S::HO) continue;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj) {
                const int tx = ix + 1 - dj;
                if (tx < 0 || (tx & 1)) continue;
                const int ox = tx >> 1;
                if (ox >= S::WO) continue;
                s += dxcol[((b * S::P) + oy * S::WO + ox) * S::KP + (di * 3 + dj) * S::CIN + ci];
            }
        }
        du_prev[i] = __float2bfloat16_rn(__bfloat162float(act[i]) > 0.f ? s : 0.f);
    }
}

// conv backward-weights on CUDA cores: dW[co][k] += sum_r dU[r][co] Xcol[r][k],
// db[co] += sum_r dU[r][co]; rows in chunks of 64 staged in shared memory.
struct ConvWgtArgs {
    const uint8_t* thumbs;
    const int32_t* prev;
    const int32_t* cur;
    const __nv_bfloat16* x;    // layers 2, 3: NHWC input
    const __nv_bfloat16* du;   // [rows][COUT]
    float* gw;                 // grad + kW
    float* gb;                 // grad + kB
    int64_t pairs;
};

template <int L>
__global__ void __launch_bounds__(256) conv_bwd_weight(const __grid_constant__ ConvWgtArgs a) {
    using S = Shape<L>;
    constexpr int R = 64, NOUT = S::COUT * S::K, PER = (NOUT + 255) / 256;
    extern __shared__ __align__(16) float wsm[];
    float* xs = wsm;                 // [R][K]
    float* us = wsm + R * S::K;      // [R][COUT]
    float acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0.f;
    float bacc = 0.f;
    const int tid = threadIdx.x;
    const int64_t rows = a.pairs * S::P;
    for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * R; r0 < rows; r0 += static_cast<int64_t>(gridDim.x) * R) {
        __syncthreads();
        for (int e = tid; e < R * S::K; e += 256) {
            const int rr = e / S::K, k = e % S::K;
            const int64_t r = r0 + rr;
            float v = 0.f;
            if (r < rows) {
                const int64_t b = r / S::P;
                const int pos = static_cast<int>(r - b * S::P);
                const int oy = pos / S::WO, ox = pos % S::WO;
                const int tap = k / S::CIN, c = k % S::CIN;
                const int iy = 2 * oy - 1 + tap / 3, ix = 2 * ox - 1 + tap % 3;
                if (iy >= 0 && iy < S::HIN && ix >= 0 && ix < S::WIN) {
                    if constexpr (L == 1) {
                        const int fi = c == 0 ? (a.prev ? a.prev[b] : static_cast<int>(b))
                                              : (a.cur ? a.cur[b] : static_cast<int>(b + 1));
                        v = (static_cast<float>(a.thumbs[static_cast<int64_t>(fi) * 2304 + iy * 64 + ix]) - 128.f) *
                            (1.f / 64.f);
                    } else {
                        v = __bfloat162float(a.x[((b * S::HIN + iy) * S::WIN + ix) * S::CIN + c]);
                    }
                }
            }
            xs[e] = v;
        }
        for (int e = tid; e < R * S::COUT; e += 256) {
            const int64_t r = r0 + e / S::COUT;
            us[e] = r < rows ? __bfloat162float(a.du[r * S::COUT + e % S::COUT]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int o = tid + 256 * i;
            if (o < NOUT) {
                const int co = o / S::K, k = o % S::K;
                float s = acc[i];
                for (int rr = 0; rr < R; ++rr) s = fmaf(us[rr * S::COUT + co], xs[rr * S::K + k], s);
                acc[i] = s;
            }
        }
        if (tid < S::COUT) {
            for (int rr = 0; rr < R; ++rr) bacc += us[rr * S::COUT + tid];
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int o = tid + 256 * i;
        if (o < NOUT) {
            const int co = o / S::K, k = o % S::K;
            const int tap = k / S::CIN, ci = k % S::CIN;
            atomicAdd(a.gw + (co * S::CIN + ci) * 9 + tap, acc[i]);
        }
    }
    if (tid < S::COUT) atomicAdd(a.gb + tid, bacc);
}

// Adam (bias-corrected), fp32 master weights
__global__ void adam_update(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <int L>
scn_status launch_bwd_data(const ConvBwdArgs& a, cudaStream_t st) {
    static int attr_dev = -1;
    int dev = 0;
    SCN_CUDA_TRY(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_bwd_data_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          BwdSmem<L>::BYTES));
        attr_dev = dev;
    }
    const int64_t tiles = (a.pairs * Shape<L>::P + 127) / 128;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    // 256 TMEM columns per CTA: at most 2 CTAs per SM can hold them
    const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(sms) * 2));
    conv_bwd_data_tc<L><<<grid, 128, BwdSmem<L>::BYTES, st>>>(a);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

template <int L>
scn_status launch_bwd_weight(const ConvWgtArgs& a, cudaStream_t st) {
    using S = Shape<L>;
    constexpr int smem = (64 * S::K + 64 * S::COUT) * 4;
    static int attr_dev = -1;
    int dev = 0;
    SCN_CUDA_TRY(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_bwd_weight<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_dev = dev;
    }
    const int64_t chunks = (a.pairs * S::P + 63) / 64;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    const int grid = static_cast<int>(std::min<int64_t>(chunks, static_cast<int64_t>(sms) * 2));
    conv_bwd_weight<L><<<grid, 256, smem, st>>>(a);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

template <int L>
scn_status launch_col2im(const float* dxcol, const __nv_bfloat16* act, __nv_bfloat16* du_prev, int64_t pairs,
                         cudaStream_t st) {
    using S = Shape<L>;
    const int64_t total = pairs * S::HIN * S::WIN * S::CIN;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 148 * 8);
    col2im_mask<L><<<static_cast<unsigned>(blocks), 256, 0, st>>>(dxcol, act, du_prev, pairs);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

// Gradients of the mean loss over one batch into n->grad (oracle layout) and n->loss.
scn_status gradients(Net* n, const uint8_t* thumbs, const int32_t* prev, const int32_t* cur, const float* labels,
                     int64_t pairs, float pos_weight, cudaStream_t st) {
    SCN_CUDA_TRY(cudaMemsetAsync(n->grad, 0, kNParams * 4, st));
    SCN_CUDA_TRY(cudaMemsetAsync(n->loss, 0, 4, st));
    scn_status s = forward_chunk(n, thumbs, prev, cur, pairs, n->z, true, st);
    if (s != SCN_OK) return s;
    const int64_t hb = std::min<int64_t>((pairs + 7) / 8, 64);
    head_bwd<<<static_cast<unsigned>(hb), 256, 0, st>>>(n->z, labels, n->g, n->v, n->a3, n->f1b, n->f2b, pos_weight,
                                                        pairs, n->grad, n->du3, n->loss);
    SCN_CUDA_TRY(cudaGetLastError());
    // layer 3
    ConvWgtArgs w{};
    w.thumbs = thumbs;
    w.prev = prev;
    w.cur = cur;
    w.pairs = pairs;
    w.x = n->a2;
    w.du = n->du3;
    w.gw = n->grad + kW3;
    w.gb = n->grad + kB3;
    if ((s = launch_bwd_weight<3>(w, st)) != SCN_OK) return s;
    ConvBwdArgs d{};
    d.pairs = pairs;
    d.status = n->status;
    d.du = n->du3;
    d.wt = n->w3t;
    d.dxcol = n->dx3;
    if ((s = launch_bwd_data<3>(d, st)) != SCN_OK) return s;
    if ((s = launch_col2im<3>(n->dx3, n->a2, n->du2, pairs, st)) != SCN_OK) return s;
    // layer 2
    w.x = n->a1;
    w.du = n->du2;
    w.gw = n->grad + kW2;
    w.gb = n->grad + kB2;
    if ((s = launch_bwd_weight<2>(w, st)) != SCN_OK) return s;
    d.du = n->du2;
    d.wt = n->w2t;
    d.dxcol = n->dx2;
    if ((s = launch_bwd_data<2>(d, st)) != SCN_OK) return s;
    if ((s = launch_col2im<2>(n->dx2, n->a1, n->du1, pairs, st)) != SCN_OK) return s;
    // layer 1 (weights only)
    w.x = nullptr;
    w.du = n->du1;
    w.gw = n->grad + kW1;
    w.gb = n->grad + kB1;
    return launch_bwd_weight<1>(w, st);
}

scn_status prep(Net* n, cudaStream_t st) {
    prep_weights<<<(32 * 288 + 255) / 256, 256, 0, st>>>(n->master, n->w1b, n->w2b, n->w3b, n->w2t, n->w3t, n->f1b,
                                                         n->f2b);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // namespace cnn
}  // namespace scn

struct scn_cnn {
    scn::cnn::Net net;
};

using namespace scn;
using namespace scn::cnn;

extern "C" {

int64_t scn_cnn_num_params(void) { return kNParams; }

scn_status scn_cnn_create(int64_t max_batch, scn_cnn** out) {
    if (!out || max_batch < 1 || max_batch > (int64_t(1) << 24)) return SCN_EINVAL;
    *out = nullptr;
    scn_cnn* c = new (std::nothrow) scn_cnn;
    if (!c) return SCN_ENOMEM;
    Net& n = c->net;
    std::memset(&n, 0, sizeof(n));
    n.max_batch = max_batch;
    const int64_t B = max_batch;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> parts = {
        {reinterpret_cast<void**>(&n.master), kNParams * 4}, {reinterpret_cast<void**>(&n.adam_m), kNParams * 4},
        {reinterpret_cast<void**>(&n.adam_v), kNParams * 4}, {reinterpret_cast<void**>(&n.grad), kNParams * 4},
        {reinterpret_cast<void**>(&n.w1b), 16 * 32 * 2},    {reinterpret_cast<void**>(&n.w2b), 32 * 144 * 2},
        {reinterpret_cast<void**>(&n.w3b), 32 * 288 * 2},   {reinterpret_cast<void**>(&n.w2t), 144 * 32 * 2},
        {reinterpret_cast<void**>(&n.w3t), 288 * 32 * 2},   {reinterpret_cast<void**>(&n.f1b), 64 * 32 * 2},
        {reinterpret_cast<void**>(&n.f2b), 64 * 2},
        {reinterpret_cast<void**>(&n.a1), size_t(B) * 576 * 16 * 2},
        {reinterpret_cast<void**>(&n.a2), size_t(B) * 144 * 32 * 2},
        {reinterpret_cast<void**>(&n.a3), size_t(B) * 40 * 32 * 2},
        {reinterpret_cast<void**>(&n.g), size_t(B) * 32 * 4},  {reinterpret_cast<void**>(&n.v), size_t(B) * 64 * 4},
        {reinterpret_cast<void**>(&n.z), size_t(B) * 4},
        {reinterpret_cast<void**>(&n.du1), size_t(B) * 576 * 16 * 2},
        {reinterpret_cast<void**>(&n.du2), size_t(B) * 144 * 32 * 2},
        {reinterpret_cast<void**>(&n.du3), size_t(B) * 40 * 32 * 2},
        {reinterpret_cast<void**>(&n.dx2), size_t(B) * 144 * 144 * 4},
        {reinterpret_cast<void**>(&n.dx3), size_t(B) * 40 * 288 * 4},
        {reinterpret_cast<void**>(&n.loss), 256}, {reinterpret_cast<void**>(&n.status), 256}};
    for (auto& p : parts) off += up(p.second);
    cudaError_t e = cudaMalloc(&n.block, off);
    if (e == cudaSuccess) e = cudaMemset(n.block, 0, off);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        if (n.block) cudaFree(n.block);
        delete c;
        return SCN_ECUDA;
    }
    char* base = static_cast<char*>(n.block);
    off = 0;
    for (auto& p : parts) {
        *p.first = base + off;
        off += up(p.second);
    }
    *out = c;
    return SCN_OK;
}

scn_status scn_cnn_destroy(scn_cnn* c) {
    if (!c) return SCN_EINVAL;
    if (c->net.block) cudaFree(c->net.block);
    delete c;
    return SCN_OK;
}

scn_status scn_cnn_set_params(scn_cnn* c, const float* h_params, int64_t n) {
    if (!c || !h_params || n != kNParams) return SCN_EINVAL;
    Net& net = c->net;
    SCN_CUDA_TRY(cudaMemcpy(net.master, h_params, kNParams * 4, cudaMemcpyHostToDevice));
    SCN_CUDA_TRY(cudaMemset(net.adam_m, 0, kNParams * 4));
    SCN_CUDA_TRY(cudaMemset(net.adam_v, 0, kNParams * 4));
    net.step = 0;
    const scn_status s = prep(&net, nullptr);
    if (s != SCN_OK) return s;
    SCN_CUDA_TRY(cudaDeviceSynchronize());
    return SCN_OK;
}

scn_status scn_cnn_get_params(const scn_cnn* c, float* h_params, int64_t n) {
    if (!c || !h_params || n != kNParams) return SCN_EINVAL;
    SCN_CUDA_TRY(cudaMemcpy(h_params, c->net.master, kNParams * 4, cudaMemcpyDeviceToHost));
    return SCN_OK;
}

scn_status scn_cnn_forward(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                           int64_t n, float* d_logits, void* stream) {
    if (!c || n < 0) return SCN_EINVAL;
    if (n == 0) return SCN_OK;
    if (!d_thumbs || !d_logits || (!d_prev) != (!d_cur)) return SCN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int64_t o = 0; o < n; o += c->net.max_batch) {
        const int64_t m = std::min<int64_t>(c->net.max_batch, n - o);
        // consecutive pairs (no index arrays): pair b of this chunk is (o + b, o + b + 1)
        const uint8_t* th = d_prev ? d_thumbs : d_thumbs + o * 2304;
        const scn_status s = forward_chunk(&c->net, th, d_prev ? d_prev + o : nullptr, d_cur ? d_cur + o : nullptr, m,
                                           d_logits + o, false, st);
        if (s != SCN_OK) return s;
    }
    return SCN_OK;
}

scn_status scn_cnn_gradients(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                             const float* d_labels, int64_t batch, float pos_weight, float* d_loss, float* d_grads,
                             void* stream) {
    if (!c || !d_thumbs || !d_labels || batch < 1 || batch > c->net.max_batch || (!d_prev) != (!d_cur))
        return SCN_EINVAL;
    if (!(pos_weight > 0.f)) return SCN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const scn_status s = gradients(&c->net, d_thumbs, d_prev, d_cur, d_labels, batch, pos_weight, st);
    if (s != SCN_OK) return s;
    if (d_grads) SCN_CUDA_TRY(cudaMemcpyAsync(d_grads, c->net.grad, kNParams * 4, cudaMemcpyDeviceToDevice, st));
    if (d_loss) SCN_CUDA_TRY(cudaMemcpyAsync(d_loss, c->net.loss, 4, cudaMemcpyDeviceToDevice, st));
    return SCN_OK;
}

scn_status scn_cnn_train_step(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                              const float* d_labels, int64_t batch, float pos_weight, float lr, float* d_loss,
                              void* stream) {
    if (!(lr > 0.f)) return SCN_EINVAL;
    const scn_status s = scn_cnn_gradients(c, d_thumbs, d_prev, d_cur, d_labels, batch, pos_weight, d_loss, nullptr,
                                           stream);
    if (s != SCN_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Net& n = c->net;
    n.step += 1;
    const float c1 = 1.f - static_cast<float>(std::pow(0.9, static_cast<double>(n.step)));
    const float c2 = 1.f - static_cast<float>(std::pow(0.999, static_cast<double>(n.step)));
    adam_update<<<(kNParams + 255) / 256, 256, 0, st>>>(n.master, n.adam_m, n.adam_v, n.grad, kNParams, lr, 0.9f,
                                                        0.999f, 1e-8f, c1, c2);
    SCN_CUDA_TRY(cudaGetLastError());
    return prep(&n, st);
}

scn_status scn_cnn_activation(const scn_cnn* c, int32_t layer, const void** d_ptr) {
    if (!c || !d_ptr) return SCN_EINVAL;
    switch (layer) {
        case 1: *d_ptr = c->net.a1; return SCN_OK;
        case 2: *d_ptr = c->net.a2; return SCN_OK;
        case 3: *d_ptr = c->net.a3; return SCN_OK;
        default: return SCN_ERANGE;
    }
}

scn_status scn_cnn_sync_status(scn_cnn* c, void* stream) {
    if (!c) return SCN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    SCN_CUDA_TRY(cudaMemcpyAsync(&h, c->net.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCN_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        SCN_CUDA_TRY(cudaMemsetAsync(c->net.status, 0, sizeof(int), st));
        SCN_CUDA_TRY(cudaStreamSynchronize(st));
        return SCN_ETIMEOUT;
    }
    return SCN_OK;
}

}  // extern "C"
