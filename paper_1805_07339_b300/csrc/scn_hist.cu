// Fused BT.601 convert + 3x16-bin histogram + shot score over a sampled
// sequence of NV12 frames, one persistent launch.
//
// What it computes (per sampled element k, frame slot[k]):
//   R = clamp((298(Y-16) + 409(V-128) + 128) >> 8, 0, 255)
//   G = clamp((298(Y-16) - 100(U-128) - 208(V-128) + 128) >> 8, 0, 255)
//   B = clamp((298(Y-16) + 516(U-128) + 128) >> 8, 0, 255)
//   hist[k][c][v >> 4] counts pixels (chroma: nearest 2x2 sample)    (Sec. 5.1.2, HIST)
//   score[k] = sum |hist[k] - hist[k-1]|, score[0] = 0;               (Sec. 3.2 stencil,
//   flag[k] = 2*score[k] > W*H                                          Sec. 5.2 shots)
//
// Design (B300):
//  * one CTA per SM; a producer warp streams each work item (a slice of rows of
//    one frame) through kStages shared-memory chunks with 1-D bulk copies
//    (TMA engine), completion on mbarriers; 8 consumer warps convert and count.
//  * the bin never needs a clamp: with x = 16*(298Y + k_c) + offset the value
//    x >> 16 is an "extended" bin in [0, rows_c) covering every byte triple, and
//    the out-of-range extended bins fold into bins 0 and 15 when the table is
//    flushed (clamp(x >> 8) >> 4 == clamp(x >> 12, 0, 15)).
//  * per pixel and channel: one dp2a (byte select + multiply + add of the
//    chroma term), one prmt (builds the shared address from the bin byte and
//    the lane's column) and one shared-memory atomic add.  Each lane owns a
//    column of its warp's table ([row][lane], 256-byte rows shared by two
//    warps), so the atomics never conflict on a bank.
//  * a slice's counts are reduced across lanes and warps, written as a
//    partial; the CTA completing a frame sums its partials into hist[k]; the
//    CTA completing the second frame of a consecutive pair computes that
//    pair's score.  Completion uses counters, nobody waits for another CTA.
#include <cuda_runtime.h>

#include <algorithm>

#include "scn_internal.h"
#include "scn_ptx.cuh"

namespace scn {
namespace {

// Extended-bin rows per channel and the offset that makes them non-negative:
// x_c >> 12 spans [-14, 30] (R), [-11, 27] (G), [-18, 33] (B) over all bytes.
constexpr int kRowsR = 45, kRowsG = 39, kRowsB = 52;
constexpr int kBaseR = 0, kBaseG = kRowsR, kBaseB = kRowsR + kRowsG;
constexpr int kOffR = 14, kOffG = 11, kOffB = 18;
static_assert(kRowsR + kRowsG + kRowsB == kTabRowsPerPair, "table rows");

// x_c = 4768*Y + K_c, K_c = 16*(chroma term + 128 - 298*16 + off_c*4096) + row base
// 4768 = 298*16; chroma weights *16: 409 -> 6544, 516 -> 8256, -100 -> -1600, -208 -> -3328.
constexpr uint32_t kWY = 4768u;
constexpr uint32_t kWV_R = 6544u;
constexpr uint32_t kWU_B = 8256u;
constexpr int32_t kWU_G = -1600, kWV_G = -3328;
constexpr int32_t kCR = 16 * (-409 * 128 + 128 - 298 * 16 + kOffR * 4096);             // 5632
constexpr int32_t kCB = 16 * (-516 * 128 + 128 - 298 * 16 + kOffB * 4096);             // 48640
constexpr int32_t kCG = 16 * (100 * 128 + 208 * 128 + 128 - 298 * 16 + kOffG * 4096);  // 1277440
static_assert(kCR == 5632 && kCB == 48640 && kCG == 1277440, "chroma constants");

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

struct HistArgs {
    const uint8_t* nv12;
    int64_t stride;
    int W, H;
    const int32_t* slot;
    int64_t n;
    int slices, rows_per_slice, chunk_rows, stage_bytes;
    uint32_t* hist;
    uint32_t* score;
    uint8_t* flag;
    uint32_t* partial;
    uint32_t* done;
    uint32_t* pair;
    int* status;
    int64_t pixel_count;
};

struct Smem {
    uint8_t* base;
    uint8_t* stages;
    uint32_t* acc;      // [2][48]
    uint64_t* full;     // [kStages]
    uint64_t* empty;    // [kStages]
    int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* smem, int stage_bytes) {
    Smem s;
    s.base = smem;
    s.stages = smem + kTabBytes;
    s.acc = reinterpret_cast<uint32_t*>(s.stages + kStages * stage_bytes);
    s.full = reinterpret_cast<uint64_t*>(s.acc + 96);
    s.empty = s.full + kStages;
    s.abort_flag = reinterpret_cast<int*>(s.empty + kStages);
    return s;
}

__device__ __forceinline__ void fail(const HistArgs& a, const Smem& s) {
    *reinterpret_cast<volatile int*>(s.abort_flag) = 1;
    atomicOr(a.status, kStatusTimeout);
}

__device__ __forceinline__ bool aborted(const Smem& s) {
    return *reinterpret_cast<volatile int*>(s.abort_flag) != 0;
}

// ---------------------------------------------------------------------------
// producer: one thread issues the bulk copies of every chunk of every item
// ---------------------------------------------------------------------------
__device__ void produce(const HistArgs& a, const Smem& s) {
    const int64_t items = a.n * a.slices;
    uint32_t it = 0, issued = 0;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t k = item / a.slices;
        const int sl = static_cast<int>(item - k * a.slices);
        const uint8_t* frame = a.nv12 + static_cast<int64_t>(a.slot[k]) * a.stride;
        const int r0 = sl * a.rows_per_slice;
        const int r1 = min(r0 + a.rows_per_slice, a.H);
        for (int r = r0; r < r1; r += a.chunk_rows, ++it) {
            const int rows = min(a.chunk_rows, r1 - r);
            const uint32_t st = it % kStages;
            if (it >= static_cast<uint32_t>(kStages) && !aborted(s)) {
                if (!ptx::mbar_wait_bounded(&s.empty[st], ((it / kStages) - 1) & 1u, kWaitLimitNs)) fail(a, s);
            }
            if (aborted(s)) continue;
            uint8_t* dst = s.stages + st * a.stage_bytes;
            const uint32_t by = static_cast<uint32_t>(rows) * a.W;
            const uint32_t buv = by / 2;
            ptx::mbar_arrive_expect_tx(&s.full[st], by + buv);
            ptx::bulk_g2s(dst, frame + static_cast<int64_t>(r) * a.W, by, &s.full[st]);
            ptx::bulk_g2s(dst + a.chunk_rows * a.W, frame + static_cast<int64_t>(a.W) * a.H + (r / 2) * a.W, buv,
                          &s.full[st]);
            issued = it + 1;
        }
    }
    // Let every copy this CTA issued land before the CTA can exit (copies stop
    // being issued after an abort, so chunks [0, issued) are the issued ones).
    for (uint32_t j = issued > kStages ? issued - kStages : 0; j < issued; ++j) {
        if (!ptx::mbar_wait_bounded(&s.full[j % kStages], (j / kStages) & 1u, kWaitLimitNs)) {
            fail(a, s);
            break;
        }
    }
}

// ---------------------------------------------------------------------------
// consumers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void count3(uint8_t* tab, uint32_t lanereg, uint32_t xr, uint32_t xg, uint32_t xb) {
    // address = (x >> 16) * 256 + lane column; byte 0 from lanereg, bytes 2,3 of x -> bytes 1,2
    atomicAdd(reinterpret_cast<uint32_t*>(tab + ptx::prmt(xr, lanereg, 0x5324u)), 1u);
    atomicAdd(reinterpret_cast<uint32_t*>(tab + ptx::prmt(xg, lanereg, 0x5324u)), 1u);
    atomicAdd(reinterpret_cast<uint32_t*>(tab + ptx::prmt(xb, lanereg, 0x5324u)), 1u);
}

// 32 pixels: 16 columns of two luma rows sharing 8 chroma samples.
__device__ __forceinline__ void count_unit(uint8_t* tab, uint32_t lanereg, uint32_t cR, uint32_t cG, uint32_t cB,
                                           uint4 y0, uint4 y1, uint4 uv) {
    const uint32_t yw0[4] = {y0.x, y0.y, y0.z, y0.w};
    const uint32_t yw1[4] = {y1.x, y1.y, y1.z, y1.w};
    const uint32_t uvw[4] = {uv.x, uv.y, uv.z, uv.w};
    const uint32_t aY0 = kWY, aY1 = kWY << 16;
    const uint32_t aR = kWV_R << 16;
    const uint32_t aB = kWU_B;
    const uint32_t aG = (static_cast<uint32_t>(kWU_G) & 0xFFFFu) | (static_cast<uint32_t>(kWV_G) << 16);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        // chroma sample (bytes 0,1) serves luma bytes 0,1; (bytes 2,3) serves luma bytes 2,3
        {
            const uint32_t kr = ptx::dp2a_lo_uu(aR, uvw[w], cR);
            const uint32_t kb = ptx::dp2a_lo_uu(aB, uvw[w], cB);
            const uint32_t kg = static_cast<uint32_t>(ptx::dp2a_lo_su(aG, uvw[w], static_cast<int32_t>(cG)));
            count3(tab, lanereg, ptx::dp2a_lo_uu(aY0, yw0[w], kr), ptx::dp2a_lo_uu(aY0, yw0[w], kg),
                   ptx::dp2a_lo_uu(aY0, yw0[w], kb));
            count3(tab, lanereg, ptx::dp2a_lo_uu(aY1, yw0[w], kr), ptx::dp2a_lo_uu(aY1, yw0[w], kg),
                   ptx::dp2a_lo_uu(aY1, yw0[w], kb));
            count3(tab, lanereg, ptx::dp2a_lo_uu(aY0, yw1[w], kr), ptx::dp2a_lo_uu(aY0, yw1[w], kg),
                   ptx::dp2a_lo_uu(aY0, yw1[w], kb));
            count3(tab, lanereg, ptx::dp2a_lo_uu(aY1, yw1[w], kr), ptx::dp2a_lo_uu(aY1, yw1[w], kg),
                   ptx::dp2a_lo_uu(aY1, yw1[w], kb));
        }
        {
            const uint32_t kr = ptx::dp2a_hi_uu(aR, uvw[w], cR);
            const uint32_t kb = ptx::dp2a_hi_uu(aB, uvw[w], cB);
            const uint32_t kg = static_cast<uint32_t>(ptx::dp2a_hi_su(aG, uvw[w], static_cast<int32_t>(cG)));
            count3(tab, lanereg, ptx::dp2a_hi_uu(aY0, yw0[w], kr), ptx::dp2a_hi_uu(aY0, yw0[w], kg),
                   ptx::dp2a_hi_uu(aY0, yw0[w], kb));
            count3(tab, lanereg, ptx::dp2a_hi_uu(aY1, yw0[w], kr), ptx::dp2a_hi_uu(aY1, yw0[w], kg),
                   ptx::dp2a_hi_uu(aY1, yw0[w], kb));
            count3(tab, lanereg, ptx::dp2a_hi_uu(aY0, yw1[w], kr), ptx::dp2a_hi_uu(aY0, yw1[w], kg),
                   ptx::dp2a_hi_uu(aY0, yw1[w], kb));
            count3(tab, lanereg, ptx::dp2a_hi_uu(aY1, yw1[w], kr), ptx::dp2a_hi_uu(aY1, yw1[w], kg),
                   ptx::dp2a_hi_uu(aY1, yw1[w], kb));
        }
    }
}

// Sum this warp's lane columns row by row, fold extended bins, add into acc[48],
// and leave the table zeroed.
__device__ __forceinline__ void flush_table(uint8_t* tab, int pair, int half, int lane, uint32_t* acc) {
    for (int t = lane; t < kTabRowsPerPair; t += 32) {
        uint8_t* row = tab + (pair * kTabRowsPerPair + t) * 256 + half * 128;
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            uint4* q = reinterpret_cast<uint4*>(row + ((lane + i) & 7) * 16);
            const uint4 v = *q;
            sum += v.x + v.y + v.z + v.w;
            *q = make_uint4(0, 0, 0, 0);
        }
        int c, e, off;
        if (t < kBaseG) { c = 0; e = t - kBaseR; off = kOffR; }
        else if (t < kBaseB) { c = 1; e = t - kBaseG; off = kOffG; }
        else { c = 2; e = t - kBaseB; off = kOffB; }
        const int b = min(max(e - off, 0), 15);
        if (sum) atomicAdd(&acc[c * 16 + b], sum);
    }
}

// Score of element k from its histogram (h0: bins lane, h1: bins 32+lane) and
// its predecessor's, read from global memory.
__device__ __forceinline__ void write_score(const HistArgs& a, int64_t k, uint32_t h0, uint32_t h1,
                                            const uint32_t* other, int lane) {
    const uint32_t p0 = ptx::ld_cg_u32(other + lane);
    const uint32_t p1 = lane < 16 ? ptx::ld_cg_u32(other + 32 + lane) : 0u;
    uint32_t d = (h0 > p0 ? h0 - p0 : p0 - h0);
    if (lane < 16) d += (h1 > p1 ? h1 - p1 : p1 - h1);
    const uint32_t s = __reduce_add_sync(0xffffffffu, d);
    if (lane == 0) {
        a.score[k] = s;
        a.flag[k] = (2ull * s > static_cast<uint64_t>(a.pixel_count)) ? 1 : 0;
    }
}

// After the consumer barrier: publish this slice, complete frames and scores.
__device__ void complete_item(const HistArgs& a, int64_t k, int sl, uint32_t* acc, int lane) {
    const uint32_t v0 = acc[lane];
    const uint32_t v1 = lane < 16 ? acc[32 + lane] : 0u;
    acc[lane] = 0;
    if (lane < 16) acc[32 + lane] = 0;
    uint32_t h0 = v0, h1 = v1;
    bool complete = true;
    if (a.slices > 1) {
        uint32_t* pp = a.partial + (k * a.slices + sl) * 48;
        pp[lane] = v0;
        if (lane < 16) pp[32 + lane] = v1;
        __threadfence();
        __syncwarp();
        uint32_t old = 0;
        if (lane == 0) old = atomicAdd(&a.done[k], 1u);
        old = __shfl_sync(0xffffffffu, old, 0);
        complete = (old == static_cast<uint32_t>(a.slices - 1));
        if (complete) {
            __threadfence();
            h0 = 0;
            h1 = 0;
            for (int j = 0; j < a.slices; ++j) {
                const uint32_t* q = a.partial + (k * a.slices + j) * 48;
                h0 += ptx::ld_cg_u32(q + lane);
                if (lane < 16) h1 += ptx::ld_cg_u32(q + 32 + lane);
            }
            if (lane == 0) a.done[k] = 0;
        }
    }
    if (!complete) return;
    a.hist[k * 48 + lane] = h0;
    if (lane < 16) a.hist[k * 48 + 32 + lane] = h1;
    if (!a.score) return;
    __threadfence();
    __syncwarp();
    if (k == 0) {
        if (lane == 0) {
            a.score[0] = 0;
            a.flag[0] = 0;
        }
    } else {
        uint32_t old = 0;
        if (lane == 0) old = atomicAdd(&a.pair[k], 1u);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old == 1) {
            __threadfence();
            write_score(a, k, h0, h1, a.hist + (k - 1) * 48, lane);
            if (lane == 0) a.pair[k] = 0;
        }
    }
    if (k + 1 < a.n) {
        uint32_t old = 0;
        if (lane == 0) old = atomicAdd(&a.pair[k + 1], 1u);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old == 1) {
            __threadfence();
            write_score(a, k + 1, h0, h1, a.hist + (k + 1) * 48, lane);
            if (lane == 0) a.pair[k + 1] = 0;
        }
    }
}

__device__ void consume(const HistArgs& a, const Smem& s, int warp, int lane) {
    const int ctid = warp * 32 + lane;
    constexpr int NT = kConsumerWarps * 32;
    const int pair = warp >> 1, half = warp & 1;
    const uint32_t lanereg = static_cast<uint32_t>(lane * 4 + half * 128);
    const uint32_t rowbase = static_cast<uint32_t>(pair * kTabRowsPerPair) << 16;
    const uint32_t cR = static_cast<uint32_t>(kCR) + rowbase + (static_cast<uint32_t>(kBaseR) << 16);
    const uint32_t cG = static_cast<uint32_t>(kCG) + rowbase + (static_cast<uint32_t>(kBaseG) << 16);
    const uint32_t cB = static_cast<uint32_t>(kCB) + rowbase + (static_cast<uint32_t>(kBaseB) << 16);
    const int W = a.W;
    const int wv = W / 16;
    const int sp = NT / wv, sc = NT % wv;
    uint8_t* tab = s.base;
    const int64_t items = a.n * a.slices;
    uint32_t it = 0;
    int rot = 0;
    int buf = 0;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t k = item / a.slices;
        const int sl = static_cast<int>(item - k * a.slices);
        const int r0 = sl * a.rows_per_slice;
        const int r1 = min(r0 + a.rows_per_slice, a.H);
        for (int r = r0; r < r1; r += a.chunk_rows, ++it) {
            const int rows = min(a.chunk_rows, r1 - r);
            const uint32_t st = it % kStages;
            if (!aborted(s)) {
                if (!ptx::mbar_wait_bounded(&s.full[st], (it / kStages) & 1u, kWaitLimitNs)) fail(a, s);
            }
            const uint8_t* ybuf = s.stages + st * a.stage_bytes;
            const uint8_t* uvbuf = ybuf + a.chunk_rows * W;
            const int units = (rows / 2) * wv;
            int u = ctid - rot;
            if (u < 0) u += NT;
            int p = u / wv;
            int c = u - p * wv;
            for (; u < units; u += NT) {
                const uint8_t* yp = ybuf + (2 * p) * W + 16 * c;
                const uint4 y0 = *reinterpret_cast<const uint4*>(yp);
                const uint4 y1 = *reinterpret_cast<const uint4*>(yp + W);
                const uint4 uv = *reinterpret_cast<const uint4*>(uvbuf + p * W + 16 * c);
                count_unit(tab, lanereg, cR, cG, cB, y0, y1, uv);
                c += sc;
                p += sp;
                if (c >= wv) {
                    c -= wv;
                    ++p;
                }
            }
            rot = (rot + units) % NT;
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.empty[st]);
        }
        uint32_t* acc = s.acc + buf * 48;
        __syncwarp();
        flush_table(tab, pair, half, lane, acc);
        ptx::named_bar_sync(1, NT);
        if (warp == 0) complete_item(a, k, sl, acc, lane);
        buf ^= 1;
    }
}

__global__ void __launch_bounds__(kHistThreads, 1) hist_kernel(HistArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const Smem s = carve(smem, a.stage_bytes);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kTabBytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid < 96) s.acc[tid] = 0;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&s.full[i], 1);
            ptx::mbar_init(&s.empty[i], kConsumerWarps);
        }
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0) produce(a, s);
        return;
    }
    consume(a, s, warp, lane);
}

// One warp per element: score[k] from hist[k-1], hist[k].
__global__ void scores_kernel(const uint32_t* hist, int64_t n, int64_t pixel_count, uint32_t* score, uint8_t* flag) {
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    if (k >= n) return;
    uint32_t d = 0;
    if (k > 0) {
        const uint32_t* h = hist + k * 48;
        const uint32_t* g = h - 48;
        const uint32_t a0 = h[lane], b0 = g[lane];
        d = a0 > b0 ? a0 - b0 : b0 - a0;
        if (lane < 16) {
            const uint32_t a1 = h[32 + lane], b1 = g[32 + lane];
            d += a1 > b1 ? a1 - b1 : b1 - a1;
        }
    }
    const uint32_t s = __reduce_add_sync(0xffffffffu, d);
    if (lane == 0) {
        score[k] = s;
        flag[k] = (2ull * s > static_cast<uint64_t>(pixel_count)) ? 1 : 0;
    }
}

bool g_attr_set = false;

}  // namespace

HistShape resolve_hist_shape(const scn_seq* s) {
    HistShape sh;
    const int W = s->table->W, H = s->table->H;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    // chunk rows: largest even count whose NV12 bytes fit one stage
    int cr = s->tune.chunk_rows;
    const int cr_max = std::max(2, (kStageBudget / (W * 3 / 2)) & ~1);
    if (cr <= 0 || cr > cr_max) cr = cr_max;
    cr = std::min(cr, H);
    // slices: enough items to keep every CTA busy with a small tail
    int slices = s->tune.slices;
    const int64_t n = std::max<int64_t>(s->n, 1);
    if (slices <= 0) {
        slices = 1;
        double best = 0.0;
        for (int c = 1; c <= s->max_slices; ++c) {
            const int64_t items = n * c;
            const int64_t rounds = (items + sms - 1) / sms;
            const double eff = static_cast<double>(items) / static_cast<double>(rounds * sms);
            if (eff > best + 0.02) {
                best = eff;
                slices = c;
            }
            if (eff >= 0.97) break;
        }
    }
    slices = std::min(slices, std::max(1, H / 2));
    int rps = ((H / 2 + slices - 1) / slices) * 2;
    slices = (H + rps - 1) / rps;
    sh.slices = slices;
    sh.rows_per_slice = rps;
    sh.chunk_rows = cr;
    const int64_t items = n * slices;
    int grid = s->tune.grid > 0 ? s->tune.grid : sms;
    sh.grid = static_cast<int>(std::min<int64_t>(grid, items));
    sh.stage_bytes = ((cr * W * 3 / 2) + 127) & ~127;
    sh.smem = static_cast<size_t>(kTabBytes) + static_cast<size_t>(kStages) * sh.stage_bytes + kSmemMisc;
    return sh;
}

static scn_status run_hist(scn_seq* s, uint32_t* d_hist, uint32_t* d_score, uint8_t* d_flag, void* stream) {
    if (!s || !d_hist) return SCN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_hist) & 3u) || (d_score && (reinterpret_cast<uintptr_t>(d_score) & 3u)))
        return SCN_EINVAL;
    if (s->n == 0) return SCN_OK;
    const HistShape sh = resolve_hist_shape(s);
    if (sh.smem > static_cast<size_t>(kSmemLimit)) return SCN_EUNSUPPORTED;
    if (!g_attr_set) {
        SCN_CUDA_TRY(cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        g_attr_set = true;
    }
    HistArgs a;
    a.nv12 = s->table->d_nv12;
    a.stride = s->table->frame_stride;
    a.W = s->table->W;
    a.H = s->table->H;
    a.slot = s->d_slot;
    a.n = s->n;
    a.slices = sh.slices;
    a.rows_per_slice = sh.rows_per_slice;
    a.chunk_rows = sh.chunk_rows;
    a.stage_bytes = sh.stage_bytes;
    a.hist = d_hist;
    a.score = d_score;
    a.flag = d_flag;
    a.partial = s->d_partial;
    a.done = s->d_done;
    a.pair = s->d_pair;
    a.status = s->d_status;
    a.pixel_count = static_cast<int64_t>(a.W) * a.H;
    hist_kernel<<<sh.grid, kHistThreads, sh.smem, static_cast<cudaStream_t>(stream)>>>(a);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // namespace scn

extern "C" {

scn_status scn_hist(scn_seq* s, uint32_t* d_hist, void* stream) {
    return scn::run_hist(s, d_hist, nullptr, nullptr, stream);
}

scn_status scn_hist_scores(scn_seq* s, uint32_t* d_hist, uint32_t* d_score, uint8_t* d_flag, void* stream) {
    if (!d_score || !d_flag) return SCN_EINVAL;
    return scn::run_hist(s, d_hist, d_score, d_flag, stream);
}

scn_status scn_shot_scores(const uint32_t* d_hist, int64_t n, int64_t pixel_count, uint32_t* d_score,
                           uint8_t* d_flag, void* stream) {
    if (n < 0 || pixel_count < 0) return SCN_EINVAL;
    if (n == 0) return SCN_OK;
    if (!d_hist || !d_score || !d_flag) return SCN_EINVAL;
    const int warps = 8;
    const int64_t blocks = (n + warps - 1) / warps;
    if (blocks > 0x7fffffff) return SCN_ERANGE;
    scn::scores_kernel<<<static_cast<unsigned>(blocks), warps * 32, 0, static_cast<cudaStream_t>(stream)>>>(
        d_hist, n, pixel_count, d_score, d_flag);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // extern "C"
