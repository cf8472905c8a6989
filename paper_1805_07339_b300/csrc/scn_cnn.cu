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
//  * conv backward-weights: tcgen05 GEMM dW^T = Xcol^T dU with the contraction
//    over all rows of the batch (pairs x output positions), operands staged
//    MN-major from the forward's im2col chunks and the rows of dU, the bias
//    gradient from a column of ones; accumulated in TMEM per CTA.
//  * head forward/backward, Adam: CUDA cores.
// Every kernel is launched as a programmatic dependent of the one before it
// (launch_pdl) and starts with pdl_wait, ahead of any global memory access and
// TMEM allocation, so a training step's 13 launches overlap one another's ends.
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
static_assert(kW1 % 4 == 0 && kW2 % 4 == 0 && kW3 % 4 == 0 && kF1 % 4 == 0 && kC1 % 4 == 0 && kF2 % 4 == 0,
              "parameter blocks added with vector atomics start on 16-byte boundaries");

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
    float* f1t;             // [32][64]  F1 as used by the forward (BF16 values), transposed
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
    uint64_t test_wait_ns;      // test hook (scn_cnn_set_wait_test): bounded-wait limit of the inference kernel
    int32_t test_withhold;      //   (0: default) and the batch whose X1 the builders withhold (< 0: none)
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
    float* zero;              // non-null: zero[0, nzero) and *zero_one set to 0 by the launch (a training
    int32_t nzero;            // step's gradient and loss accumulators, ahead of every kernel that adds to them)
    float* zero_one;
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

// Threads that gather each 128-row tile of the training convolutions: every one of a
// thread's im2col loads is in flight before its first store; layers with many k chunks per
// row (2 and 3) split each row over four threads, layer 1 (four chunks) keeps one.
template <int L>
constexpr int gather_parts() { return Shape<L>::KP / 8 >= 16 ? 4 : 1; }

template <int L>
__global__ void __launch_bounds__(128 * gather_parts<L>()) conv_fwd_tc(const __grid_constant__ ConvFwdArgs a) {
    constexpr int kConvParts = gather_parts<L>(), kConvThreads = 128 * kConvParts;
    ptx::pdl_wait();
    ptx::pdl_release();
    if (a.zero) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nzero; i += gridDim.x * blockDim.x) a.zero[i] = 0.f;
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.zero_one = 0.f;
    }
    using S = Shape<L>;
    using M = ConvSmem<L>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* As = smem;
    uint8_t* Bs = smem + M::A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + M::A_BYTES + M::B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & 127, part = tid >> 7;  // the tile row this thread gathers, and which of its k chunks
    // weights -> B tile (core layout), once
    for (int e = tid; e < S::COUT * (S::KP / 8); e += kConvThreads) {
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
    constexpr int NJ = (S::KP / 8 + kConvParts - 1) / kConvParts;  // k chunks per thread
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // A tile: k chunks part, part + kConvParts, ... of row `row`, loads first
        const int64_t r = t * 128 + row;
        const bool live = r < rows;
        const int64_t b = live ? r / S::P : 0;
        const int pos = live ? static_cast<int>(r - b * S::P) : 0;
        uint4 v[NJ];
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
            const int j = part + q * kConvParts;
            v[q] = (live && j < S::KP / 8) ? im2col_chunk<L>(a, b, pos, j) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
            const int j = part + q * kConvParts;
            if (j < S::KP / 8) *reinterpret_cast<uint4*>(As + tc::core_offset(row, 8 * j, S::KP)) = v[q];
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
        // epilogue by warps 0-3: thread = row, COUT columns
        if (warp < 4) {
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
    // F1 as fp32 in shared memory, row pitch 33 (a warp reading column c of 32 rows hits 32 banks)
    __shared__ float sf1[64 * 33];
    ptx::pdl_wait();
    ptx::pdl_release();
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) sf1[(i >> 5) * 33 + (i & 31)] = __bfloat162float(f1b[i]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    if (b >= pairs) return;
    float s = 0.f;
    const __nv_bfloat16* p = a3 + b * 40 * 32 + lane;
    __nv_bfloat16 av[40];  // every load in flight before the (ordered) sum
#pragma unroll
    for (int pos = 0; pos < 40; ++pos) av[pos] = p[pos * 32];
#pragma unroll
    for (int pos = 0; pos < 40; ++pos) s += __bfloat162float(av[pos]);
    const float g = s * (1.f / 40.f);
    float v0 = c1[lane], v1 = c1[lane + 32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const float gc = __shfl_sync(0xffffffffu, g, c);
        v0 = fmaf(sf1[lane * 33 + c], gc, v0);
        v1 = fmaf(sf1[(lane + 32) * 33 + c], gc, v1);
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
                             __nv_bfloat16* w2t, __nv_bfloat16* w3t, __nv_bfloat16* f1b, __nv_bfloat16* f2b,
                             float* f1t) {
    ptx::pdl_wait();
    ptx::pdl_release();
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
    if (i < 64 * 32) f1t[(i % 32) * 64 + i / 32] = __bfloat162float(__float2bfloat16_rn(m[kF1 + i]));
}

template <int L>
scn_status launch_conv_fwd(const ConvFwdArgs& a, cudaStream_t st) {
    static std::atomic<uint64_t> attr_done{0};
    const scn_status sa = once_per_device(attr_done, [] {
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_fwd_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          ConvSmem<L>::BYTES));
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_fwd_tc<L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        return SCN_OK;
    });
    if (sa != SCN_OK) return sa;
    const int64_t tiles = (a.pairs * Shape<L>::P + 127) / 128;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(sms) * 4));
    SCN_CUDA_TRY(launch_pdl(conv_fwd_tc<L>, dim3(grid), dim3(128 * gather_parts<L>()), ConvSmem<L>::BYTES, st, a));
    return SCN_OK;
}

// forward of one chunk of at most max_batch pairs; keeps head intermediates when train is set
scn_status forward_chunk(Net* n, const uint8_t* thumbs, const int32_t* prev, const int32_t* cur, int64_t pairs,
                         float* logits, bool train, cudaStream_t st) {
    ConvFwdArgs a{};
    if (train) {  // the gradient and loss accumulators, zeroed by the first launch of the step
        a.zero = n->grad;
        a.nzero = kNParams;
        a.zero_one = n->loss;
    }
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
    a.zero = nullptr;
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
    SCN_CUDA_TRY(launch_pdl(head_fwd, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, st, n->a3, n->f1b,
                            n->master + kC1, n->f2b, n->master + kC2, train ? n->g : nullptr,
                            train ? n->v : nullptr, logits, pairs));
    return SCN_OK;
}

// ---------------------------------------------------------------------------
// fused forward (inference): per-batch activation layouts in shared memory
// ---------------------------------------------------------------------------
// The inference kernel below takes kFzPairs pairs (a batch) at a time and keeps
// every activation in shared memory.  Each convolution is an implicit GEMM whose A operand the tensor core
// reads straight out of the activation buffer, one filter tap per MMA (no
// im2col copy): the buffers are laid out so that, for a fixed tap, the 8-row
// core matrices of the output positions sit at one constant stride.  Stride 2
// is absorbed by keeping even and odd input columns (for layer 1 also even and
// odd input rows) in separate planes; the zero padding of the convolutions is
// stored as explicit zero rows and entries.  One "entry" is 8 bf16 (16 bytes):
// 8 channels of one pixel, or for layer 1 the 2 channels of 3 neighbouring
// columns plus 2 zeros.
//
// Tiles are 16 groups of 8 output positions (M = 128).  Groups are enumerated
// so that consecutive groups are consecutive output rows (layer 1: 4 groups per
// row); the last tile of a layer starts at G - 16 and keeps only the groups it
// adds, and group slots past a pair's last output row are computed and dropped.
constexpr int kFzPairs = 2;
// layer 1 input X1: planes O1 (odd input rows; row 0 of a pair = zero padding
// above the image) and E1 (even input rows; row 18 of a pair = zeros); a plane
// row holds the 32 output columns ox, entry ox = [prev, cur] at input columns
// 2ox-1, 2ox, 2ox+1, then 2 zeros
constexpr int kFzR1 = 19;
constexpr int kFzX1Rows = kFzPairs * kFzR1 + 1;
constexpr int kFzX1Plane = kFzX1Rows * 512;
constexpr int kFzG1 = kFzPairs * kFzR1 * 4;
constexpr int kFzT1 = (kFzG1 + 15) / 16;
// layer 2 input A1 (a1, 16 channels = 2 chunks): per chunk an even-column plane
// (16 entries per row, entry m = column 2m) and an odd-column plane (17 entries,
// entry u = column 2u-1, entry 0 = zero padding); row 0 of a pair = zero padding,
// rows 1..18 = a1 rows, row 19 spare
constexpr int kFzR2 = 20;
constexpr int kFzA1Rows = kFzPairs * kFzR2 + 1;
constexpr int kFzE2Pitch = 16 * 16, kFzO2Pitch = 17 * 16;
constexpr int kFzE2Plane = kFzA1Rows * kFzE2Pitch, kFzO2Plane = kFzA1Rows * kFzO2Pitch;
constexpr int kFzG2 = kFzPairs * 10;  // groups per column half (9 output rows + 1 dropped)
// layer 3 input A2 (a2, 32 channels = 4 chunks): even plane 8 entries, odd plane
// 9 entries; row 0 of each pair and row kFzPairs*10 = zero padding (row 10 of a
// pair is row 0 of the next).  Dropped groups read past a plane into the next
// one or past the last one; every such read stays inside the A2 buffer (kFzF1T).
constexpr int kFzR3 = 10;
constexpr int kFzA2Rows = kFzPairs * kFzR3 + 1;
constexpr int kFzE3Pitch = 8 * 16, kFzO3Pitch = 9 * 16;
constexpr int kFzE3Plane = kFzA2Rows * kFzE3Pitch, kFzO3Plane = kFzA2Rows * kFzO3Pitch;
constexpr int kFzA2Bytes = 4 * (kFzE3Plane + kFzO3Plane);
constexpr int kFzG3 = kFzPairs * 5;
constexpr int kFzF1T = 24576;  // end of what layer 3's dropped groups read of the A2 buffer
constexpr int kFzReg0Bytes = 2 * kFzX1Plane;                    // X1
constexpr int kFzReg1Bytes = 2 * kFzE2Plane + 2 * kFzO2Plane;   // A1
static_assert(kFzG1 >= 16 && kFzG2 >= 16, "every layer-1/2 tile lies inside the buffers");
// every row the MMAs read lies inside its plane (layers 1, 2) or inside the A2 buffer (layer 3)
static_assert((kFzG1 - 1) / 4 + 1 < kFzX1Rows, "layer-1 reads");
static_assert(2 * (kFzG2 - 1) + 2 < kFzA1Rows, "layer-2 reads");
static_assert(4 * kFzE3Plane + 3 * kFzO3Plane + (2 * 15 + 2 + 1) * kFzO3Pitch <= kFzF1T, "layer-3 reads");
static_assert(kFzA2Bytes <= kFzF1T, "A2 buffer");
static_assert(kFzPairs == 2, "the head's warp split (warp 12 + p: pair p) and the zero-row layout assume two pairs");

struct FusedArgs {
    const uint8_t* thumbs;
    const int32_t* prev;      // null: pair b = (b, b + 1)
    const int32_t* cur;
    int64_t pairs;
    const __nv_bfloat16* w1b;  // [16][32], k = tap*2 + c
    const __nv_bfloat16* w2b;  // [32][144], k = tap*16 + ci
    const __nv_bfloat16* w3b;  // [32][288], k = tap*32 + ci
    const float* master;       // fp32 parameters (biases)
    const __nv_bfloat16* f1b;
    const __nv_bfloat16* f2b;
    const float* f1t;          // [32][64] fp32 (BF16 values), transposed F1
    float* logits;
    int* status;
    const int* d_pairs;        // non-null: the pair count, read on the device (at most pairs)
    const int32_t* out_index;  // non-null: pair b's logit goes to logits[out_index[b]]
    uint64_t wait_ns;          // bounded-wait limit (test hook; 0 = kWaitNs)
    int32_t withhold;          // test hook: the builders withhold X1 of this local batch (< 0: none)
};

// (byte k of w - 128) / 64 as fp32: the byte placed in the mantissa of 2^23
// (one prmt) gives 2^23 + byte exactly; one fma scales and shifts it, exactly
// (the result needs 23 significant bits at most)
template <int K>
__device__ __forceinline__ float thumb_at(const uint32_t (&w)[8]) {
    const uint32_t m = ptx::prmt(w[K >> 2], 0x4B000000u, 0x7540u | (K & 3));
    return fmaf(__uint_as_float(m), 1.f / 64.f, -(8388608.f / 64.f + 2.f));
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void fz_sync() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// ---------------------------------------------------------------------------
// inference: warp-specialised pipeline over batches, one CTA per SM
// ---------------------------------------------------------------------------
// Four warp groups of four warps work on different batches at the same time,
// each on buffers of its own, and hand each batch on through mbarriers:
//   group 0 (warps 0-3):   X1 of batch j and its conv1 MMAs;
//   group 1 (warps 4-7):   conv1 epilogue of batch j into A1[j & 1];
//   group 2 (warps 8-11):  conv2 of batch j (MMAs and epilogue) into A2[j & 1];
//   group 3 (warps 12-15): conv3 of batch j (warp 15 issues its MMAs, one batch
//                          ahead), pooling and the head (FC1, FC2).
// A batch then takes the time of the slowest group, not the sum of the phases.
// Each layer's MMAs are issued by lane 0 of several warps of the group that
// produces its input (conv1) or consumes its output (conv2, conv3), so no
// layer waits behind another's in an issue queue: one thread issues one
// accumulating tcgen05.mma per ~145 cycles (each waits for the one before,
// whatever accumulator it writes), while 2 and 4 issuing threads reach 74 and
// 41 cycles per MMA of 128 x 32 x 16 (measured on the B300).  The per-batch
// layouts are those above; X1 is single, A1 and A2 double-buffered, and their
// padding is written once.  conv1's bias enters through the MMA (every X1
// entry carries 1.0 in its two spare K slots, W1 holds the bias split into two
// BF16 parts there, so the epilogue is one conversion with ReLU per two
// values); conv2 accumulates all 9 taps in one accumulator per tile, conv3 its
// two K halves in two.  Each group owns the four TMEM lane quadrants through
// its four warps; TMEM holds conv1's accumulators twice (columns 0-159 and
// 160-319, batch parity), conv2's at 320-447, conv3's at 448-511.  Every wait
// is bounded (2 s), after which the thread records a timeout and stops
// waiting; no thread leaves its loop early, so every barrier is still reached.
constexpr int kPpThreads = 512;
constexpr int kPpW1 = 0;                                   // [16][32]
constexpr int kPpW2 = kPpW1 + 16 * 32 * 2;                 // 9 x [32][16]
constexpr int kPpW3 = kPpW2 + 9 * 32 * 16 * 2;             // 9 x [32][32]
constexpr int kPpBias = kPpW3 + 9 * 32 * 32 * 2;           // floats: b1 16, b2 32, b3 32, c1 64, f2 64, c2 1
// mbarriers (count): X1 built (128 builder threads), X1 read by conv1 (4
// issuers), conv1 tile done (2 TMEM buffers x 10 tiles, 1 each), conv1 TMEM
// buffer read by group 1 (2, 4 warps each), A1[b] written (128), A1[b] read by
// conv2 (4 issuers), conv2 tile done (4, 1 each), A2[b] written (128), A2[b]
// read by conv3 (1 issuer), conv3 done (1 issuer).  Groups 2 and 3 reuse their
// TMEM accumulators after a group barrier that follows their warps' reads;
// group 0 issues conv1 into a buffer that group 1 has released.
constexpr int kBX1Full = 0, kBX1Free = 1, kBT1Full = 2, kBT1Free = kBT1Full + 2 * kFzT1, kBA1Full = kBT1Free + 2,
              kBA1Free = kBA1Full + 2,
              kBT2Full = kBA1Free + 2, kBA2Full = kBT2Full + 4, kBA2Free = kBA2Full + 2, kBT3Full = kBA2Free + 2,
              kPpNBar = kBT3Full + 1;
constexpr int kPpT1 = 0, kPpT2 = 2 * kFzT1 * 16, kPpT3 = kPpT2 + 4 * 32;  // TMEM columns (conv3: 2 x 32)
constexpr int kPpBar = kPpBias + 1024;
constexpr int kPpX1 = (kPpBar + kPpNBar * 8 + 16 + 1023) / 1024 * 1024;  // O1, E1 planes
constexpr int kPpA1 = kPpX1 + kFzReg0Bytes;                               // 2 x A1
constexpr int kPpA2Bytes = kFzF1T;  // A2 and what its dropped groups read beyond it
constexpr int kPpA2 = kPpA1 + 2 * kFzReg1Bytes;                           // 2 x A2
constexpr int kPpPart = kPpA2 + 2 * kPpA2Bytes;                           // 2 x [pair][5][32] fp32
constexpr int kPpF1 = kPpPart + 2 * kFzPairs * 5 * 32 * 4;                // F1 transposed, [32][64] fp32
constexpr int kPpSmem = kPpF1 + 32 * 64 * 4;
constexpr int kPpTmemCols = 512;
constexpr uint32_t kPpOnes = 0x3F803F80u;  // BF16 1.0 in both halves: X1's bias slots
static_assert(kPpT3 + 64 <= kPpTmemCols, "TMEM columns");
static_assert(kPpSmem <= 232448, "one CTA per SM");
static_assert(kFzReg1Bytes % 16 == 0 && kPpA2Bytes % 16 == 0 && kFzReg0Bytes % 16 == 0, "16-byte buffers");
static_assert(kFzPairs * 36 % 4 == 0, "build rows split evenly over the four builder warps");

// bounded wait by one thread (no warp-wide step: callers may be a single lane)
__device__ __forceinline__ bool pp_wait1(uint64_t* bar, uint32_t par, bool ok, int* status, uint64_t limit) {
    if (ok && !ptx::mbar_wait_bounded(bar, par, limit)) {
        atomicOr(status, kStatusTimeout);
        ok = false;
    }
    return ok;
}

__device__ __forceinline__ void pp_group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void pp_group_sync96(int id) { asm volatile("bar.sync %0, 96;" ::"r"(id) : "memory"); }

// max(lo, 0) and max(hi, 0) rounded to BF16 (round to nearest even), packed lo | hi << 16
__device__ __forceinline__ uint32_t relu_pack(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__global__ void __launch_bounds__(kPpThreads, 1) cnn_forward_pipe(const __grid_constant__ FusedArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp >> 2, quad = warp & 3;
    const int r = 32 * quad + lane;  // TMEM lane = tile row of this thread in the epilogues
    float* bias = reinterpret_cast<float*>(smem + kPpBias);  // b1 @0, b2 @16, b3 @48, c1 @80, f2 @144, c2 @208
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kPpBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kPpBar + kPpNBar * 8);
    uint8_t* X1 = smem + kPpX1;
    const uint32_t sbase = ptx::smem_u32(smem);
    // launched behind the previous kernel of the stream (thumbnails, list): wait for it
    // before the first global read; the next kernel may be scheduled from here on
    ptx::pdl_wait();
    ptx::pdl_release();

    // ---- once: weights, biases, zeroed activation buffers, barriers, TMEM.  Every global
    //      load is issued first (one round trip to L2 for all of them), the buffers are zeroed
    //      while they are in flight, then the values are stored in their layouts.
    static_assert(32 * 64 == 4 * kPpThreads, "F1: four entries per thread");
    uint4 w2r[2], w3r[3];
    float f1r[4];
#pragma unroll
    for (int i = 0; i < 2; ++i) {  // W2: tap x 32 rows x 2 entries
        const int e = tid + i * kPpThreads, t = e / 64, n = (e >> 1) & 31, j = e & 1;
        if (e < 9 * 32 * 2) w2r[i] = __ldg(reinterpret_cast<const uint4*>(a.w2b + n * 144 + t * 16 + 8 * j));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {  // W3: tap x 32 rows x 4 entries
        const int e = tid + i * kPpThreads, t = e / 128, n = (e >> 2) & 31, j = e & 3;
        if (e < 9 * 32 * 4) w3r[i] = __ldg(reinterpret_cast<const uint4*>(a.w3b + n * 288 + t * 32 + 8 * j));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) f1r[i] = a.f1t[tid + i * kPpThreads];
    // biases: b1 @0, b2 @16, b3 @48, c1 @80, f2 @144, c2 @208 (thread tid loads entry tid of each)
    const float rb1 = tid < 16 ? a.master[kB1 + tid] : 0.f;
    const float rb2 = tid < 32 ? a.master[kB2 + tid] : 0.f, rb3 = tid < 32 ? a.master[kB3 + tid] : 0.f;
    const float rc1 = tid < 64 ? a.master[kC1 + tid] : 0.f;
    const float rf2 = tid < 64 ? __bfloat162float(a.f2b[tid]) : 0.f;
    const float rc2 = tid == 0 ? a.master[kC2] : 0.f;
    // W1: 16 rows x 4 entries of 8 K slots, thread e < 64 builds entry e; conv1's bias sits in
    // the K slots 6 and 7 of the first filter row, as two BF16 parts whose sum is the fp32
    // bias to 16 significant bits (X1 carries 1.0 there)
    uint16_t w1h[8];
    float w1b1 = 0.f;
    if (tid < 16 * 4) {
        const int n = tid >> 2, j = tid & 3;
        w1b1 = a.master[kB1 + n];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 8 * j + i, dy = k >> 3, rem = k & 7, dx = rem >> 1, c = rem & 1;
            w1h[i] = (dy < 3 && rem < 6) ? __bfloat16_as_ushort(a.w1b[n * 32 + (dy * 3 + dx) * 2 + c]) : 0;
        }
    }
    // X1: every entry 0 with 1.0 in the two bias slots (the padding rows keep it: the
    // build writes the image rows only); both A1 and both A2 buffers zero (the
    // epilogues write the live entries only)
    for (int e = tid; e < kFzReg0Bytes / 16; e += kPpThreads)
        reinterpret_cast<uint4*>(X1)[e] = make_uint4(0, 0, 0, kPpOnes);
    for (int e = tid; e < (kPpPart - kPpA1) / 16; e += kPpThreads)
        reinterpret_cast<uint4*>(smem + kPpA1)[e] = make_uint4(0, 0, 0, 0);
    if (tid < 16 * 4) {
        const int n = tid >> 2, j = tid & 3;
        const __nv_bfloat16 bhi = __float2bfloat16_rn(w1b1);
        const __nv_bfloat16 blo = __float2bfloat16_rn(w1b1 - __bfloat162float(bhi));
        if (j == 0) {  // K slots 6, 7 of the first entry
            w1h[6] = __bfloat16_as_ushort(bhi);
            w1h[7] = __bfloat16_as_ushort(blo);
        }
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = static_cast<uint32_t>(w1h[2 * q]) | (static_cast<uint32_t>(w1h[2 * q + 1]) << 16);
        *reinterpret_cast<uint4*>(smem + kPpW1 + tc::core_offset(n, 8 * j, 32)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int e = tid + i * kPpThreads, t = e / 64, n = (e >> 1) & 31, j = e & 1;
        if (e < 9 * 32 * 2) *reinterpret_cast<uint4*>(smem + kPpW2 + t * 1024 + tc::core_offset(n, 8 * j, 16)) = w2r[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int e = tid + i * kPpThreads, t = e / 128, n = (e >> 2) & 31, j = e & 3;
        if (e < 9 * 32 * 4) *reinterpret_cast<uint4*>(smem + kPpW3 + t * 2048 + tc::core_offset(n, 8 * j, 32)) = w3r[i];
    }
    if (tid < 16) bias[tid] = rb1;
    if (tid < 32) {
        bias[16 + tid] = rb2;
        bias[48 + tid] = rb3;
    }
    if (tid < 64) {
        bias[80 + tid] = rc1;
        bias[144 + tid] = rf2;
    }
    if (tid == 0) bias[208] = rc2;
#pragma unroll
    for (int i = 0; i < 4; ++i) reinterpret_cast<float*>(smem + kPpF1)[tid + i * kPpThreads] = f1r[i];
    if (tid == 0) {
        for (int i = 0; i < kPpNBar; ++i) {
            uint32_t cnt = 1;  // tcgen05.commit of one issuer
            if (i == kBX1Full || i == kBA1Full || i == kBA1Full + 1 || i == kBA2Full || i == kBA2Full + 1)
                cnt = 128;  // every thread of the writing group
            else if (i == kBX1Free || i == kBA1Free || i == kBA1Free + 1 || i == kBT1Free || i == kBT1Free + 1)
                cnt = 4;  // the four conv1 (X1) or conv2 (A1) issuers, or group 1's four readers
            ptx::mbar_init(bar + i, cnt);
        }
        ptx::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, kPpTmemCols);
    fz_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tlane = static_cast<uint32_t>(32 * quad) << 16;
    bool ok = true;
    const uint64_t wlim = a.wait_ns ? a.wait_ns : kWaitNs;

    const int64_t npairs = a.d_pairs ? min(static_cast<int64_t>(max(*a.d_pairs, 0)), a.pairs) : a.pairs;
    const int64_t nbatch = (npairs + kFzPairs - 1) / kFzPairs;
    // batches of this CTA: blockIdx.x + j * gridDim.x, j < nb
    const int nb = blockIdx.x < nbatch ? static_cast<int>((nbatch - 1 - blockIdx.x) / gridDim.x + 1) : 0;

    if (grp == 0) {
        // ---- group 0: X1 of batch j (warp w builds input rows w, w + 4, ...: lane = output
        //      column, one 512-byte plane row per store)
        constexpr int kRows = kFzPairs * 36 / 4;
        const int64_t b0 = blockIdx.x;
        int64_t ip0 = 0, ic0 = 0, ip1 = 0, ic1 = 0;
        auto pair_thumbs = [&](int64_t batch, int p, int64_t& ip, int64_t& ic) {
            int64_t b = batch * kFzPairs + p;
            if (b >= npairs) b = npairs - 1;
            ip = a.prev ? a.prev[b] : b;
            ic = a.cur ? a.cur[b] : b + 1;
        };
        if (nb > 0) {
            pair_thumbs(b0, 0, ip0, ic0);
            pair_thumbs(b0, 1, ip1, ic1);
        }
        for (int j = 0; j < nb; ++j) {
            const int64_t batch = b0 + static_cast<int64_t>(j) * gridDim.x;
            uint32_t vps[kRows], vqs[kRows];
#pragma unroll
            for (int q = 0; q < kRows; ++q) {  // every load in flight before the first store
                const int task = warp + 4 * q, p = task / 36, iy = task - 36 * p;
                const int64_t ip = p ? ip1 : ip0, ic = p ? ic1 : ic0;
                vps[q] = __ldg(reinterpret_cast<const uint16_t*>(a.thumbs + ip * 2304 + iy * 64) + lane);
                vqs[q] = __ldg(reinterpret_cast<const uint16_t*>(a.thumbs + ic * 2304 + iy * 64) + lane);
            }
            if (j + 1 < nb) {  // the next batch's thumbnail indices
                pair_thumbs(batch + gridDim.x, 0, ip0, ic0);
                pair_thumbs(batch + gridDim.x, 1, ip1, ic1);
            }
            // X1 is free once the conv1 MMAs of batch j-1 have completed
            if (j > 0) ok = pp_wait1(&bar[kBX1Free], (j - 1) & 1, ok, a.status, wlim);
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int task = warp + 4 * q, p = task / 36, iy = task - 36 * p;
                const uint32_t vp = vps[q], vq = vqs[q];
                const uint32_t up = __shfl_up_sync(0xffffffffu, vp, 1), uq = __shfl_up_sync(0xffffffffu, vq, 1);
                const uint32_t w[8] = {vp, vq, up, uq, 0, 0, 0, 0};
                const uint32_t w0 = lane ? bf16x2(thumb_at<9>(w), thumb_at<13>(w)) : 0u;  // column -1 is padding
                const uint32_t w1 = bf16x2(thumb_at<0>(w), thumb_at<4>(w));
                const uint32_t w2 = bf16x2(thumb_at<1>(w), thumb_at<5>(w));
                uint8_t* row = (iy & 1) ? X1 + (p * kFzR1 + ((iy + 1) >> 1)) * 512
                                        : X1 + kFzX1Plane + (p * kFzR1 + (iy >> 1)) * 512;
                *reinterpret_cast<uint4*>(row + lane * 16) = make_uint4(w0, w1, w2, kPpOnes);
            }
            tc::fence_proxy_async();
            if (j != a.withhold) ptx::mbar_arrive(&bar[kBX1Full]);  // test hook: a withheld batch times out
            // conv1 of batch j into TMEM buffer j & 1: lane 0 of warp w issues tiles w, w + 4,
            // w + 8 once every builder is done and group 1 has read the buffer (batch j-2)
            if (lane == 0) {
                const int cb = j & 1;
                ok = pp_wait1(&bar[kBX1Full], j & 1, ok, a.status, wlim);
                if (j >= 2) ok = pp_wait1(&bar[kBT1Free + cb], ((j >> 1) + 1) & 1, ok, a.status, wlim);
                tc::fence_after_sync();
                constexpr uint32_t idesc = tc::idesc_bf16(128, 16);
                for (int t = warp; t < kFzT1; t += 4) {
                    const uint32_t g0 = static_cast<uint32_t>(min(16 * t, kFzG1 - 16));
                    const uint32_t acc = tmem + kPpT1 + 16 * (kFzT1 * cb + t);
#pragma unroll
                    for (int k = 0; k < 2; ++k)
                        tc::mma(acc, tc::smem_desc(sbase + kPpX1 + 512 * k + g0 * 128, kFzX1Plane, 128),
                                tc::smem_desc(sbase + kPpW1 + 256 * k, 128, 512), idesc, k ? 1u : 0u);
                    tc::commit(&bar[kBT1Full + kFzT1 * cb + t]);
                }
                tc::commit(&bar[kBX1Free]);
            }
            __syncwarp();
        }
    } else if (grp == 1) {
        // ---- group 1: conv1 epilogue of batch j (ReLU, BF16; the bias is in the
        //      accumulator) into A1[j & 1], four tiles (64 columns) per TMEM load
        for (int j = 0; j < nb; ++j) {
            const int b = j & 1;
            uint8_t* E2 = smem + kPpA1 + b * kFzReg1Bytes;
            uint8_t* O2 = E2 + 2 * kFzE2Plane;
            // A1[b] is free once the conv2 MMAs of batch j-2 have completed
            if (j >= 2) ok = pp_wait1(&bar[kBA1Free + b], ((j >> 1) + 1) & 1, ok, a.status, wlim);
            const uint32_t t1 = tmem + tlane + kPpT1 + 16 * kFzT1 * b;  // the batch's conv1 accumulators
            for (int t0 = 0; t0 < kFzT1; t0 += 4) {
                const int nt = min(4, kFzT1 - t0);
                for (int u = 0; u < nt; ++u)
                    ok = pp_wait1(&bar[kBT1Full + kFzT1 * b + t0 + u], (j >> 1) & 1, ok, a.status, wlim);
                __syncwarp();
                tc::fence_after_sync();
                uint32_t accs[64];
                if (nt == 4) {
                    tc::ld64(t1 + 16 * t0, accs);
                } else {
                    tc::ld32(t1 + 16 * t0, *reinterpret_cast<uint32_t(*)[32]>(accs));
                }
                tc::wait_ld();
                if (t0 + nt == kFzT1) {  // the batch's conv1 accumulators are read
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&bar[kBT1Free + b]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u >= nt) break;
                    const int t = t0 + u;
                    const uint32_t* acc = accs + 16 * u;
                    const int g0 = min(16 * t, kFzG1 - 16);
                    const int g = g0 + (r >> 3);
                    const int p = g / (kFzR1 * 4), rem = g - p * (kFzR1 * 4), oy = rem >> 2;
                    if (g >= 16 * t && oy < 18) {
                        const int ox = 8 * (rem & 3) + (r & 7);
                        uint32_t o[8];
#pragma unroll
                        for (int c = 0; c < 16; c += 2)
                            o[c / 2] = relu_pack(__uint_as_float(acc[c]), __uint_as_float(acc[c + 1]));
                        const int row = p * kFzR2 + oy + 1;
                        uint8_t* dst = (ox & 1) ? O2 + row * kFzO2Pitch + ((ox + 1) >> 1) * 16
                                                : E2 + row * kFzE2Pitch + (ox >> 1) * 16;
                        const int cs = (ox & 1) ? kFzO2Plane : kFzE2Plane;
                        *reinterpret_cast<uint4*>(dst) = make_uint4(o[0], o[1], o[2], o[3]);
                        *reinterpret_cast<uint4*>(dst + cs) = make_uint4(o[4], o[5], o[6], o[7]);
                    }
                }
            }
            tc::fence_proxy_async();
            ptx::mbar_arrive(&bar[kBA1Full + b]);
        }
    } else if (grp == 2) {
        // ---- group 2: conv2 of batch j (lane 0 of warp 8 + q issues tile q, all 9 taps),
        //      then its epilogue (bias, ReLU, BF16) into A2[j & 1]
        float b2[32];  // in registers: a broadcast 16-byte shared load costs four wavefronts
#pragma unroll
        for (int c = 0; c < 32; ++c) b2[c] = bias[16 + c];
        for (int j = 0; j < nb; ++j) {
            const int b = j & 1;
            if (j > 0) {  // every warp of the group has read batch j-1's conv2 accumulators
                tc::fence_before_sync();
                pp_group_sync(2);
                tc::fence_after_sync();
            }
            if (lane == 0) {
                ok = pp_wait1(&bar[kBA1Full + b], (j >> 1) & 1, ok, a.status, wlim);
                tc::fence_after_sync();
                constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
                // tile quad: column half h, first group g0; tap (dy, dx) reads the even-
                // column plane (dx = 1) or the odd one, shifted by one entry for dx = 2
                const int h = quad >> 1, g0 = (quad & 1) ? kFzG2 - 16 : 0;
                const uint32_t s_e2 = sbase + kPpA1 + b * kFzReg1Bytes, s_o2 = s_e2 + 2 * kFzE2Plane;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
                    const uint32_t rp = dx == 1 ? kFzE2Pitch : kFzO2Pitch;
                    const uint32_t cs = dx == 1 ? kFzE2Plane : kFzO2Plane;
                    const uint32_t ad = (dx == 1 ? s_e2 : s_o2) + (2 * g0 + dy) * rp + (8 * h + (dx == 2 ? 1 : 0)) * 16;
                    tc::mma(tmem + kPpT2 + 32 * quad, tc::smem_desc(ad, cs, 2 * rp),
                            tc::smem_desc(sbase + kPpW2 + tap * 1024, 128, 256), idesc, tap > 0 ? 1u : 0u);
                }
                tc::commit(&bar[kBT2Full + quad]);
                tc::commit(&bar[kBA1Free + b]);
            }
            __syncwarp();
            uint8_t* E3 = smem + kPpA2 + b * kPpA2Bytes;
            uint8_t* O3 = E3 + 4 * kFzE3Plane;
            if (j >= 2) ok = pp_wait1(&bar[kBA2Free + b], ((j >> 1) + 1) & 1, ok, a.status, wlim);
            for (int tt = 0; tt < 4; ++tt) {
                ok = pp_wait1(&bar[kBT2Full + tt], j & 1, ok, a.status, wlim);
                __syncwarp();
                tc::fence_after_sync();
                const int h = tt >> 1, first = (tt & 1) ? 16 : 0, g0 = (tt & 1) ? kFzG2 - 16 : 0;
                const int g = g0 + (r >> 3), p = g / 10, oy = g - 10 * p;
                const bool live = g >= first && oy < 9;
                const int ox = 8 * h + (r & 7);
                const int row = p * kFzR3 + oy + 1;
                uint8_t* dst = (ox & 1) ? O3 + row * kFzO3Pitch + ((ox + 1) >> 1) * 16
                                        : E3 + row * kFzE3Pitch + (ox >> 1) * 16;
                const int cs = (ox & 1) ? kFzO3Plane : kFzE3Plane;
                uint32_t us[32];
                tc::ld32(tmem + tlane + kPpT2 + 32 * tt, us);
                tc::wait_ld();
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    const uint32_t* u0 = us + c0;
                    if (live) {
                        uint32_t o[8];
#pragma unroll
                        for (int c = 0; c < 16; c += 2)
                            o[c / 2] = relu_pack(__uint_as_float(u0[c]) + b2[c0 + c],
                                                 __uint_as_float(u0[c + 1]) + b2[c0 + c + 1]);
                        const int q = c0 / 8;
                        *reinterpret_cast<uint4*>(dst + q * cs) = make_uint4(o[0], o[1], o[2], o[3]);
                        *reinterpret_cast<uint4*>(dst + (q + 1) * cs) = make_uint4(o[4], o[5], o[6], o[7]);
                    }
                }
            }
            tc::fence_proxy_async();
            ptx::mbar_arrive(&bar[kBA2Full + b]);
        }
    } else {
        // ---- group 3: conv3 of batch j, its epilogue (bias, ReLU, BF16 rounding), each
        //      output row's 8 positions summed by shuffles into part[j & 1], and the head
        //      (warp 12 + p: pair p's logit: mean, FC1, ReLU, FC2).  Warp 15 (its lanes hold
        //      dropped rows only) issues conv3 (both K halves, one accumulator each): batch
        //      j + 1's as soon as the group has read batch j's accumulators, so that the MMAs
        //      run while the other three warps pool and compute the head of batch j.
        auto issue_conv3 = [&](int jj) {  // lane 0 of warp 15
            const int bb = jj & 1;
            ok = pp_wait1(&bar[kBA2Full + bb], (jj >> 1) & 1, ok, a.status, wlim);
            tc::fence_after_sync();
            constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
            const uint32_t s_e3 = sbase + kPpA2 + bb * kPpA2Bytes, s_o3 = s_e3 + 4 * kFzE3Plane;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap % 3;
                const uint32_t rp = dx == 1 ? kFzE3Pitch : kFzO3Pitch;
                const uint32_t cs = dx == 1 ? kFzE3Plane : kFzO3Plane;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint32_t ad = (dx == 1 ? s_e3 : s_o3) + 2 * kk * cs + dy * rp + (dx == 2 ? 16 : 0);
                    tc::mma(tmem + kPpT3 + 32 * kk, tc::smem_desc(ad, cs, 2 * rp),
                            tc::smem_desc(sbase + kPpW3 + tap * 2048 + kk * 256, 128, 512), idesc, tap > 0 ? 1u : 0u);
                }
            }
            tc::commit(&bar[kBT3Full]);
            tc::commit(&bar[kBA2Free + bb]);
        };
        float b3r[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) b3r[c] = bias[48 + c];
        const float c1a = bias[80 + lane], c1b = bias[80 + 32 + lane];
        const float f2a = bias[144 + lane], f2b = bias[144 + 32 + lane], c2 = bias[208];
        if (quad == 3 && lane == 0 && nb > 0) issue_conv3(0);
        __syncwarp();
        for (int j = 0; j < nb; ++j) {
            const int b = j & 1;
            float* part = reinterpret_cast<float*>(smem + kPpPart) + b * (kFzPairs * 5 * 32);
            ok = pp_wait1(&bar[kBT3Full], j & 1, ok, a.status, wlim);
            __syncwarp();
            tc::fence_after_sync();
            uint32_t acc2[64];  // the two accumulators (K halves), 32 channels each
            tc::ld64(tmem + tlane + kPpT3, acc2);
            tc::wait_ld();
            tc::fence_before_sync();
            pp_group_sync(1);  // every warp has read batch j's conv3 accumulators
            tc::fence_after_sync();
            if (quad == 3) {
                if (lane == 0 && j + 1 < nb) issue_conv3(j + 1);
                __syncwarp();
                continue;
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    acc[c] = __float_as_uint(__uint_as_float(acc2[16 * half + c]) + __uint_as_float(acc2[32 + 16 * half + c]));
                const int g = r >> 3;
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    v[c] = g < kFzG3 ? __bfloat162float(__float2bfloat16_rn(
                                           fmaxf(__uint_as_float(acc[c]) + b3r[16 * half + c], 0.f)))
                                     : 0.f;
#pragma unroll
                for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
                if (g < kFzG3 && (lane & 7) == 0) {
                    const int p = g / 5, oy = g - 5 * p;
                    float4* dst = reinterpret_cast<float4*>(part + (p * 5 + oy) * 32 + 16 * half);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            pp_group_sync96(3);  // part[b] complete (warps 12-14; part[b] of batch j-2 no longer read)
            if (quad < kFzPairs) {
                const int p = quad;
                const float* q = part + p * 160 + lane;
                const float gl = (q[0] + q[32] + q[64] + q[96] + q[128]) * (1.f / 40.f);
                const float* f1 = reinterpret_cast<const float*>(smem + kPpF1);
                float v0 = c1a, v1 = c1b;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float gc = __shfl_sync(0xffffffffu, gl, c);
                    v0 = fmaf(f1[c * 64 + lane], gc, v0);
                    v1 = fmaf(f1[c * 64 + 32 + lane], gc, v1);
                }
                float z0 = f2a * fmaxf(v0, 0.f), z1 = f2b * fmaxf(v1, 0.f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    z0 += __shfl_xor_sync(0xffffffffu, z0, o);
                    z1 += __shfl_xor_sync(0xffffffffu, z1, o);
                }
                const int64_t pb = (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(j) * gridDim.x) * kFzPairs + p;
                if (lane == 0 && pb < npairs) a.logits[a.out_index ? a.out_index[pb] : pb] = z0 + z1 + c2;
            }
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kPpTmemCols);
}

scn_status launch_forward_fused(Net* n, const uint8_t* thumbs, const int32_t* prev, const int32_t* cur, int64_t pairs,
                                float* logits, cudaStream_t st, const int* d_pairs = nullptr,
                                const int32_t* out_index = nullptr) {
    static std::atomic<uint64_t> attr_done{0};
    const scn_status sa = once_per_device(attr_done, [] {
        SCN_CUDA_TRY(cudaFuncSetAttribute(cnn_forward_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, kPpSmem));
        SCN_CUDA_TRY(cudaFuncSetAttribute(cnn_forward_pipe, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        return SCN_OK;
    });
    if (sa != SCN_OK) return sa;
    FusedArgs a{};
    a.thumbs = thumbs;
    a.prev = prev;
    a.cur = cur;
    a.pairs = pairs;
    a.w1b = n->w1b;
    a.w2b = n->w2b;
    a.w3b = n->w3b;
    a.master = n->master;
    a.f1b = n->f1b;
    a.f2b = n->f2b;
    a.f1t = n->f1t;
    a.logits = logits;
    a.status = n->status;
    a.d_pairs = d_pairs;
    a.out_index = out_index;
    a.wait_ns = n->test_wait_ns;
    a.withhold = n->test_withhold;
    const int64_t nbatch = (pairs + kFzPairs - 1) / kFzPairs;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    const int grid = static_cast<int>(std::min<int64_t>(nbatch, static_cast<int64_t>(sms)));
    SCN_CUDA_TRY(launch_pdl(cnn_forward_pipe, dim3(grid), dim3(kPpThreads), kPpSmem, st, a));
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
    // F1 staged in shared memory; the block's gradient sums of F1 (row c of 65 words holds
    // column c of F1, so that both a warp's 32 rows j and 32 consecutive columns c hit 32
    // banks), c1 and F2, added by its warps and then to `grad` with 16-byte vector atomics
    constexpr int kF1s = 32 * 65;
    __shared__ __nv_bfloat16 sf1[64 * 32];
    __shared__ float sacc[kF1s + 64 + 64];
    ptx::pdl_wait();
    ptx::pdl_release();
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < 64 * 32; i += blockDim.x) sf1[i] = f1b[i];
    for (int i = tid; i < kF1s + 128; i += blockDim.x) sacc[i] = 0.f;
    __syncthreads();
    const int64_t w0 = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    float dF1a[32], dF1b[32];  // rows j = lane and lane + 32
#pragma unroll
    for (int c = 0; c < 32; ++c) dF1a[c] = dF1b[c] = 0.f;
    float dc1a = 0.f, dc1b = 0.f, dF2a = 0.f, dF2b = 0.f, dc2 = 0.f, lsum = 0.f;
    const float inv_b = 1.f / static_cast<float>(pairs);
    const float f2a = __bfloat162float(f2b[lane]), f2c = __bfloat162float(f2b[lane + 32]);
    for (int64_t b = w0; b < pairs; b += nw) {
        // the pair's a3 (for the ReLU mask of du3) requested first, with its other inputs
        uint16_t am[40];
        const uint16_t* ap = reinterpret_cast<const uint16_t*>(a3 + b * 40 * 32 + lane);
#pragma unroll
        for (int pos = 0; pos < 40; ++pos) am[pos] = ap[pos * 32];
        const float zz = z[b], yy = y[b];
        const float va = v[b * 64 + lane], vb = v[b * 64 + 32 + lane];
        const float gl = g[b * 32 + lane];
        const float sig = 1.f / (1.f + __expf(-zz));
        const float dz = (pos_weight * yy * (sig - 1.f) + (1.f - yy) * sig) * inv_b;
        // softplus(-z), softplus(z) for the loss
        const float spn = fmaxf(-zz, 0.f) + log1pf(__expf(-fabsf(zz)));
        const float spp = fmaxf(zz, 0.f) + log1pf(__expf(-fabsf(zz)));
        lsum += (pos_weight * yy * spn + (1.f - yy) * spp) * inv_b;
        const float ha = fmaxf(va, 0.f), hb = fmaxf(vb, 0.f);
        dF2a += dz * ha;
        dF2b += dz * hb;
        dc2 += dz;
        const float dva = va > 0.f ? dz * f2a : 0.f;
        const float dvb = vb > 0.f ? dz * f2c : 0.f;
        dc1a += dva;
        dc1b += dvb;
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
            dg = fmaf(__bfloat162float(sf1[j * 32 + lane]), dvj_a, dg);
            dg = fmaf(__bfloat162float(sf1[(j + 32) * 32 + lane]), dvj_b, dg);
        }
        const __nv_bfloat16 da3 = __float2bfloat16_rn(dg * (1.f / 40.f));
        const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
        __nv_bfloat16* dp = du3 + b * 40 * 32 + lane;
#pragma unroll
        for (int pos = 0; pos < 40; ++pos)  // a3 > 0: bit patterns 0x0001 (least positive) .. 0x7F80 (+inf)
            dp[pos * 32] = (static_cast<uint32_t>(am[pos]) - 1u < 0x7F80u) ? da3 : zero;
    }
    if (w0 < pairs) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            atomicAdd(&sacc[c * 65 + lane], dF1a[c]);
            atomicAdd(&sacc[c * 65 + 32 + lane], dF1b[c]);
        }
        atomicAdd(&sacc[kF1s + lane], dc1a);
        atomicAdd(&sacc[kF1s + 32 + lane], dc1b);
        atomicAdd(&sacc[kF1s + 64 + lane], dF2a);
        atomicAdd(&sacc[kF1s + 64 + 32 + lane], dF2b);
        // dc2 and the loss are the same in every lane (they depend on z only)
        if (lane == 0) {
            atomicAdd(grad + kC2, dc2);
            atomicAdd(loss, lsum);
        }
    }
    __syncthreads();
    // F1's gradient is [j][c] in `grad`: four consecutive columns c of row j per vector atomic
    for (int i = tid; i < 64 * 32 / 4; i += blockDim.x) {
        const int j = i >> 3, c = (i & 7) * 4;
        const float4 v = make_float4(sacc[c * 65 + j], sacc[(c + 1) * 65 + j], sacc[(c + 2) * 65 + j],
                                     sacc[(c + 3) * 65 + j]);
        atomicAdd(reinterpret_cast<float4*>(grad + kF1) + i, v);
    }
    if (tid < 16) {  // c1 and F2: 64 each
        atomicAdd(reinterpret_cast<float4*>(grad + kC1) + tid,
                  make_float4(sacc[kF1s + 4 * tid], sacc[kF1s + 4 * tid + 1], sacc[kF1s + 4 * tid + 2],
                              sacc[kF1s + 4 * tid + 3]));
    } else if (tid < 32) {
        const int u = tid - 16;
        atomicAdd(reinterpret_cast<float4*>(grad + kF2) + u,
                  make_float4(sacc[kF1s + 64 + 4 * u], sacc[kF1s + 64 + 4 * u + 1], sacc[kF1s + 64 + 4 * u + 2],
                              sacc[kF1s + 64 + 4 * u + 3]));
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
    static constexpr int S_OFF = A_BYTES + B_BYTES + 64;  // the epilogue's 128 x 48 staging block
    static constexpr int BYTES = S_OFF + 128 * 52 * 4;
};

template <int L>
__global__ void __launch_bounds__(128) conv_bwd_data_tc(const __grid_constant__ ConvBwdArgs a) {
    ptx::pdl_wait();
    ptx::pdl_release();
    using S = Shape<L>;
    using M = BwdSmem<L>;
    constexpr int NH = S::KP > 144 ? 2 : 1;   // N halves
    constexpr int NN = S::KP / NH;            // 144 for both layers
    static_assert(NN % 48 == 0 && NN <= 256, "N: three 16-column TMEM loads at a time");
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
    // work item w: row tile w / NH, column half w % NH (the halves of a tile run on separate CTAs)
    for (int64_t w = blockIdx.x; w < tiles * NH; w += gridDim.x) {
        const int64_t t = w / NH;
        const int h = static_cast<int>(w - t * NH);
        const int64_t r = t * 128 + tid;
        const bool live = r < rows;
#pragma unroll
        for (int j = 0; j < S::COUT / 8; ++j) {
            const uint4 v = live ? __ldg(reinterpret_cast<const uint4*>(a.du + r * S::COUT + 8 * j)) : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(As + tc::core_offset(tid, 8 * j, S::COUT)) = v;
        }
        tc::fence_proxy_async();
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
        // three 16-column TMEM loads in flight per wait; the 128 x 48 block goes through shared
        // memory (row pitch 52 floats: a quarter warp's 16-byte stores hit 8 distinct bank groups)
        // so that consecutive threads store consecutive 16-byte pieces of a row
        float* stg = reinterpret_cast<float*>(smem + M::S_OFF);
#pragma unroll 1
        for (int c0 = 0; c0 < NN; c0 += 48) {
            uint32_t q[3][16];
#pragma unroll
            for (int g = 0; g < 3; ++g) tc::ld16(tmem + ((32u * warp) << 16) + c0 + 16 * g, q[g]);
            tc::wait_ld();
            float4* srow = reinterpret_cast<float4*>(stg + tid * 52);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const uint32_t* qi = q[i >> 2] + 4 * (i & 3);
                srow[i] = make_float4(__uint_as_float(qi[0]), __uint_as_float(qi[1]), __uint_as_float(qi[2]),
                                      __uint_as_float(qi[3]));
            }
            __syncthreads();
            if (ok) {
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    const int f = tid + 128 * k, rr = f / 12, c4 = f - rr * 12;
                    const int64_t row = t * 128 + rr;
                    if (row < rows)
                        reinterpret_cast<float4*>(a.dxcol + row * S::KP + h * NN + c0)[c4] =
                            reinterpret_cast<const float4*>(stg + rr * 52)[c4];
                }
            }
            __syncthreads();
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
    ptx::pdl_wait();
    ptx::pdl_release();
    using S = Shape<L>;
    static_assert(S::CIN % 4 == 0 && S::KP % 4 == 0, "four channels per thread, 16-byte dX loads");
    constexpr int Q = S::CIN / 4;  // channel quads per input position
    // one thread per input position and channel quad (32-bit indices: the launch checks the count)
    const int total = static_cast<int>(pairs) * S::HIN * S::WIN * Q;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c4 = i % Q, q = i / Q;
    const int ix = q % S::WIN, iy = (q / S::WIN) % S::HIN, b = q / (S::WIN * S::HIN);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
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
            const float4 v = __ldg(reinterpret_cast<const float4*>(
                dxcol + (static_cast<int64_t>(b) * S::P + oy * S::WO + ox) * S::KP + (di * 3 + dj) * S::CIN + 4 * c4));
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    // ReLU mask of the layer below: its activation > 0 (bf16 bit patterns 0x0001 .. 0x7F80)
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(act) + i);
    auto pos = [](uint32_t h) { return (h & 0xFFFFu) - 1u < 0x7F80u; };
    const float r0 = pos(a.x) ? acc.x : 0.f, r1 = pos(a.x >> 16) ? acc.y : 0.f;
    const float r2 = pos(a.y) ? acc.z : 0.f, r3 = pos(a.y >> 16) ? acc.w : 0.f;
    reinterpret_cast<uint2*>(du_prev)[i] = make_uint2(pack_bf16(r0, r1), pack_bf16(r2, r3));
}

// Arguments of the backward-weights kernel.
struct ConvWgtArgs {
    const uint8_t* thumbs;
    const int32_t* prev;
    const int32_t* cur;
    const __nv_bfloat16* x;    // layers 2, 3: NHWC input
    const __nv_bfloat16* du;   // [rows][COUT]
    float* gw;                 // grad + kW
    float* gb;                 // grad + kB
    int64_t pairs;
    int* status;               // tensor-core path: bounded-wait status word
};

// conv backward-weights on tcgen05: D[k][co] = sum_r Xcol[r][k] dU[r][co] over
// the CTA's rows r (pairs x output positions), i.e. dW^T with the contraction
// over rows; row K of Xcol is set to 1 so that D[K][co] = sum_r dU[r][co] is
// the bias gradient.  M = k (tiles of 128, K + 1 rounded up), N = COUT, rows
// in chunks of 128 (8 MMAs of 16 rows per M tile).  Both operands are staged
// "MN-major" (no swizzle): a core matrix is 8 rows r x 8 consecutive k (or co)
// values, i.e. 16 contiguous bytes of one im2col or dU row, so the staging is
// the forward's im2col chunk writes and plain 16-byte copies of dU.  The
// accumulator stays in TMEM across all chunks of the CTA; the epilogue adds it
// to the fp32 gradient (oracle layout) with one atomic per element.
template <int L>
struct WgtTc {
    using S = Shape<L>;
    static constexpr int MT = (S::K + 1 + 127) / 128;   // M tiles (k, plus the ones row)
    static constexpr int MP = MT * 128;
    static constexpr int KCH = S::K / 8 + 1;             // 8-wide k chunks written per row (ones included)
    static constexpr int A_BYTES = MP * 128 * 2, B_BYTES = S::COUT * 128 * 2;
    static constexpr int BYTES = A_BYTES + B_BYTES + 64;
    static constexpr uint32_t TMEM_COLS = MT * S::COUT <= 32 ? 32 : (MT * S::COUT <= 64 ? 64 : 128);
    static_assert(MT * S::COUT <= 128, "TMEM columns");
    static_assert(S::K % 8 != 0 || S::K / 8 < MP / 8, "ones chunk inside the tile");
};
// element E of 8 packed BF16 values |= 1.0 (the element is zero before)
template <int E>
__device__ __forceinline__ void set_bf16_one(uint4& v) {
    constexpr uint32_t bits = (E & 1) ? (0x3F80u << 16) : 0x3F80u;
    if constexpr (E / 2 == 0) v.x |= bits;
    else if constexpr (E / 2 == 1) v.y |= bits;
    else if constexpr (E / 2 == 2) v.z |= bits;
    else v.w |= bits;
}

// MN-major no-swizzle descriptors: the stride between core matrices along MN
// goes in the stride-byte-offset field, the stride along K in the
// leading-byte-offset field
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t mn_stride, uint32_t k_stride) {
    return tc::smem_desc(saddr, k_stride, mn_stride);
}

// The weight-gradient kernel gathers its 128-row chunks the same way (gather_parts threads a row).
template <int L>
__global__ void __launch_bounds__(128 * gather_parts<L>()) conv_bwd_weight_tc(const __grid_constant__ ConvWgtArgs a) {
    constexpr int kWgtParts = gather_parts<L>(), kWgtThreads = 128 * kWgtParts;
    ptx::pdl_wait();
    ptx::pdl_release();
    using S = Shape<L>;
    using W = WgtTc<L>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* As = smem;                  // [r/8][MP/8] cores of 8 r x 8 k
    uint8_t* Bs = smem + W::A_BYTES;     // [r/8][COUT/8] cores of 8 r x 8 co
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + W::A_BYTES + W::B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & 127, part = tid >> 7;  // the chunk row this thread gathers, and which of its k chunks
    // k columns beyond the written chunks stay zero for the whole launch
    for (int i = tid; i < (W::A_BYTES + W::B_BYTES) / 16; i += kWgtThreads)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        ptx::mbar_init(mbar, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, W::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t a_addr = ptx::smem_u32(As), b_addr = ptx::smem_u32(Bs);
    constexpr uint32_t kAK = (W::MP / 8) * 128, kBK = (S::COUT / 8) * 128;  // K-direction core strides
    constexpr uint32_t idesc = tc::idesc_bf16(128, S::COUT) | (1u << 15) | (1u << 16);  // A, B MN-major
    // im2col arguments of the forward's staging
    ConvFwdArgs f{};
    f.thumbs = a.thumbs;
    f.prev = a.prev;
    f.cur = a.cur;
    f.x = a.x;
    const int64_t rows = a.pairs * S::P;
    const int64_t chunks = (rows + 127) / 128;
    uint32_t phase = 0;
    bool ok = true, first = true;
    constexpr int NJ = (S::KP / 8 + kWgtParts - 1) / kWgtParts;  // k chunks per thread
    constexpr int NG = (S::COUT / 8 + kWgtParts - 1) / kWgtParts;  // dU chunks per thread
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        const int64_t r = c * 128 + row;
        const bool live = r < rows;
        const int64_t b = live ? r / S::P : 0;
        const int pos = live ? static_cast<int>(r - b * S::P) : 0;
        uint8_t* arow = As + (row >> 3) * (W::MP / 8) * 128 + (row & 7) * 16;
        uint8_t* brow = Bs + (row >> 3) * (S::COUT / 8) * 128 + (row & 7) * 16;
        // k chunks part, part + kWgtParts, ... of the row and its dU chunks: loads first
        uint4 v[NJ], u[NG];
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
            const int j = part + q * kWgtParts;
            v[q] = (live && j < S::KP / 8) ? im2col_chunk<L>(f, b, pos, j) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            const int g = part + q * kWgtParts;
            u[q] = (live && g < S::COUT / 8) ? __ldg(reinterpret_cast<const uint4*>(a.du + r * S::COUT + 8 * g))
                                             : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
            const int j = part + q * kWgtParts;
            if (j < S::KP / 8) {
                if (j == S::K / 8 && live) set_bf16_one<S::K % 8>(v[q]);  // the ones column k = K shares this chunk
                *reinterpret_cast<uint4*>(arow + j * 128) = v[q];
            }
        }
        if constexpr (S::K % 8 == 0) {
            // the ones column starts its own chunk
            if (part == (S::K / 8) % kWgtParts)
                *reinterpret_cast<uint4*>(arow + (S::K / 8) * 128) =
                    live ? make_uint4(0x3F80u, 0, 0, 0) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            const int g = part + q * kWgtParts;
            if (g < S::COUT / 8) *reinterpret_cast<uint4*>(brow + g * 128) = u[q];
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int t = 0; t < W::MT; ++t) {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    tc::mma(tmem + t * S::COUT, mn_desc(a_addr + t * 16 * 128 + kk * 2 * kAK, 128, kAK),
                            mn_desc(b_addr + kk * 2 * kBK, 128, kBK), idesc, (first && kk == 0) ? 0u : 1u);
                }
            }
            tc::commit(mbar);
        }
        first = false;
        // the next chunk overwrites the operands: wait for these MMAs
        if (ok && !ptx::mbar_wait_bounded(mbar, phase, kWaitNs)) {
            ok = false;
            atomicOr(a.status, kStatusTimeout);
        }
        phase ^= 1u;
        tc::fence_after_sync();
    }
    // epilogue: warps 0-3 read the accumulators (TMEM lane = k within the tile, column = co; the
    // loads are warp-wide) and place the CTA's partial gradient in the operand buffer, free once
    // the last MMAs have completed, in the gradient's own layout [co][ci][tap]; then every thread
    // adds it to global memory with 16-byte vector atomics over contiguous words (the per-k
    // addresses are 36 bytes apart: one atomic per element would cost one transaction each)
    static_assert(S::COUT * S::K * 4 <= W::A_BYTES && (S::COUT * S::K) % 4 == 0, "partial gradient in the A buffer");
    float* pgrad = reinterpret_cast<float*>(As);
    if (!first && warp < 4) {
#pragma unroll
        for (int t = 0; t < W::MT; ++t) {
            const int k = t * 128 + tid;
#pragma unroll
            for (int c0 = 0; c0 < S::COUT; c0 += 16) {
                uint32_t q[16];
                tc::ld16(tmem + ((32u * warp) << 16) + t * S::COUT + c0, q);
                tc::wait_ld();
                if (k < S::K) {
                    const int tap = k / S::CIN, ci = k % S::CIN;
#pragma unroll
                    for (int i = 0; i < 16; ++i) pgrad[(c0 + i) * S::K + ci * 9 + tap] = __uint_as_float(q[i]);
                } else if (k == S::K && ok) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) atomicAdd(a.gb + c0 + i, __uint_as_float(q[i]));
                }
            }
        }
    }
    __syncthreads();
    if (!first && ok) {
        // the gradient block is 16-byte aligned: the parameter offsets of W1, W2, W3 are multiples of 4
        const float4* p4 = reinterpret_cast<const float4*>(pgrad);
        float4* g4 = reinterpret_cast<float4*>(a.gw);
        for (int i = tid; i < S::COUT * S::K / 4; i += blockDim.x) atomicAdd(g4 + i, p4[i]);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, W::TMEM_COLS);
}

// Adam (bias-corrected), fp32 master weights
__global__ void adam_update(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    ptx::pdl_wait();
    ptx::pdl_release();
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
    static std::atomic<uint64_t> attr_done{0};
    const scn_status sa = once_per_device(attr_done, [] {
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_bwd_data_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          BwdSmem<L>::BYTES));
        return SCN_OK;
    });
    if (sa != SCN_OK) return sa;
    const int64_t tiles = (a.pairs * Shape<L>::P + 127) / 128;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    // one work item per row tile and column half; 256 TMEM columns per CTA: at most 2 CTAs per SM
    constexpr int NH = Shape<L>::KP > 144 ? 2 : 1;
    const int grid = static_cast<int>(std::min<int64_t>(tiles * NH, static_cast<int64_t>(sms) * 2));
    SCN_CUDA_TRY(launch_pdl(conv_bwd_data_tc<L>, dim3(grid), dim3(128), BwdSmem<L>::BYTES, st, a));
    return SCN_OK;
}

template <int L>
scn_status launch_bwd_weight(const ConvWgtArgs& a, cudaStream_t st) {
    using S = Shape<L>;
    if (a.pairs <= 0) return SCN_OK;
    static std::atomic<uint64_t> attr_done{0};
    const scn_status sa = once_per_device(attr_done, [] {
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_bwd_weight_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          WgtTc<L>::BYTES));
        SCN_CUDA_TRY(cudaFuncSetAttribute(conv_bwd_weight_tc<L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        return SCN_OK;
    });
    if (sa != SCN_OK) return sa;
    const int64_t chunks = (a.pairs * S::P + 127) / 128;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    // as many CTAs per SM as shared memory and threads allow (at most 4: TMEM columns fit)
    constexpr int threads = 128 * gather_parts<L>();
    const int per_sm = std::max(1, std::min<int>(std::min(4, 2048 / threads), (227 * 1024) / (WgtTc<L>::BYTES + 1024)));
    const int grid = static_cast<int>(std::min<int64_t>(chunks, static_cast<int64_t>(sms) * per_sm));
    SCN_CUDA_TRY(launch_pdl(conv_bwd_weight_tc<L>, dim3(grid), dim3(threads), WgtTc<L>::BYTES, st, a));
    return SCN_OK;
}

template <int L>
scn_status launch_col2im(const float* dxcol, const __nv_bfloat16* act, __nv_bfloat16* du_prev, int64_t pairs,
                         cudaStream_t st) {
    using S = Shape<L>;
    // one thread per input position and four channels: every thread's loads in flight at once
    const int64_t total = pairs * S::HIN * S::WIN * (S::CIN / 4);
    if (total > 0x7fffffff) return SCN_ERANGE;
    const int64_t blocks = (total + 255) / 256;
    SCN_CUDA_TRY(
        launch_pdl(col2im_mask<L>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, st, dxcol, act, du_prev, pairs));
    return SCN_OK;
}

// Gradients of the mean loss over one batch into n->grad (oracle layout) and n->loss.
scn_status gradients(Net* n, const uint8_t* thumbs, const int32_t* prev, const int32_t* cur, const float* labels,
                     int64_t pairs, float pos_weight, cudaStream_t st) {
    scn_status s = forward_chunk(n, thumbs, prev, cur, pairs, n->z, true, st);  // zeroes grad and loss
    if (s != SCN_OK) return s;
    const int64_t hb = std::min<int64_t>((pairs + 7) / 8, 64);
    SCN_CUDA_TRY(launch_pdl(head_bwd, dim3(static_cast<unsigned>(hb)), dim3(256), 0, st, n->z, labels, n->g, n->v,
                            n->a3, n->f1b, n->f2b, pos_weight, pairs, n->grad, n->du3, n->loss));
    // layer 3
    ConvWgtArgs w{};
    w.thumbs = thumbs;
    w.prev = prev;
    w.cur = cur;
    w.pairs = pairs;
    w.status = n->status;
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
    SCN_CUDA_TRY(launch_pdl(prep_weights, dim3((32 * 288 + 255) / 256), dim3(256), 0, st, n->master, n->w1b, n->w2b,
                            n->w3b, n->w2t, n->w3t, n->f1b, n->f2b, n->f1t));
    return SCN_OK;
}

}  // namespace cnn
}  // namespace scn

struct scn_cnn {
    scn::cnn::Net net;
};

namespace scn {
scn_status cnn_forward_counted(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                               int64_t max_pairs, const int* d_pairs, float* d_logits, cudaStream_t st,
                               const int32_t* d_out_index) {
    if (!c || !d_thumbs || !d_prev || !d_cur || !d_pairs || !d_logits || max_pairs < 0) return SCN_EINVAL;
    if (max_pairs == 0) return SCN_OK;
    if (reinterpret_cast<uintptr_t>(d_thumbs) % 16) return SCN_EINVAL;
    return cnn::launch_forward_fused(&c->net, d_thumbs, d_prev, d_cur, max_pairs, d_logits, st, d_pairs, d_out_index);
}
}  // namespace scn

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
    n.test_wait_ns = 0;    // the test hook off: default wait limit,
    n.test_withhold = -1;  // nothing withheld
    const int64_t B = max_batch;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> parts = {
        {reinterpret_cast<void**>(&n.master), kNParams * 4}, {reinterpret_cast<void**>(&n.adam_m), kNParams * 4},
        {reinterpret_cast<void**>(&n.adam_v), kNParams * 4}, {reinterpret_cast<void**>(&n.grad), kNParams * 4},
        {reinterpret_cast<void**>(&n.w1b), 16 * 32 * 2},    {reinterpret_cast<void**>(&n.w2b), 32 * 144 * 2},
        {reinterpret_cast<void**>(&n.w3b), 32 * 288 * 2},   {reinterpret_cast<void**>(&n.w2t), 144 * 32 * 2},
        {reinterpret_cast<void**>(&n.w3t), 288 * 32 * 2},   {reinterpret_cast<void**>(&n.f1b), 64 * 32 * 2},
        {reinterpret_cast<void**>(&n.f2b), 64 * 2},    {reinterpret_cast<void**>(&n.f1t), 32 * 64 * 4},
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
    if (reinterpret_cast<uintptr_t>(d_thumbs) % 16) return SCN_EINVAL;  // rows are read as 16-byte vectors
    return launch_forward_fused(&c->net, d_thumbs, d_prev, d_cur, n, d_logits, static_cast<cudaStream_t>(stream));
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
    SCN_CUDA_TRY(launch_pdl(adam_update, dim3((kNParams + 255) / 256), dim3(256), 0, st, n.master, n.adam_m,
                            n.adam_v, n.grad, kNParams, lr, 0.9f, 0.999f, 1e-8f, c1, c2));
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

scn_status scn_cnn_set_wait_test(scn_cnn* c, uint64_t wait_limit_ns, int32_t withhold_batch) {
    if (!c) return SCN_EINVAL;
    if (wait_limit_ns != 0 && (wait_limit_ns < 100000ull || wait_limit_ns > 10000000000ull)) return SCN_EINVAL;
    c->net.test_wait_ns = wait_limit_ns;
    c->net.test_withhold = withhold_batch < 0 ? -1 : withhold_batch;
    return SCN_OK;
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
