// Fused BT.601 convert + 3x16-bin histogram + shot score over sampled
// sequences of NV12 frames, one persistent launch for one sequence or for a
// batch of sequences of different tables and resolutions.
//
// What it computes (per sampled element k of a sequence, frame slot[k]):
//   R = clamp((298(Y-16) + 409(V-128) + 128) >> 8, 0, 255)
//   G = clamp((298(Y-16) - 100(U-128) - 208(V-128) + 128) >> 8, 0, 255)
//   B = clamp((298(Y-16) + 516(U-128) + 128) >> 8, 0, 255)
//   hist[k][c][v >> 4] counts pixels (chroma: nearest 2x2 sample)    (Sec. 5.1.2, HIST)
//   score[k] = sum |hist[k] - hist[k-1]|, score[0] = 0;               (Sec. 3.2 stencil,
//   flag[k] = 2*score[k] > W*H                                          Sec. 5.2 shots)
//
// Design (B300):
//  * Work queue: the work is a list of items, each a range of "row pairs" (two
//    luma rows and the chroma row they share) of one frame of one sequence
//    (the paper's work packets, Sec. 4.1).  Each CTA's producer warp pops items
//    with an atomic counter; the last CTA to find the queue empty resets it, so
//    a launch leaves the counters zero and needs no memset (graph replays too).
//  * One CTA per SM: the producer warp walks the CTA's work and hands out
//    chunk descriptors (sequence, element, first row, rows) through a small
//    mbarrier ring; 20 consumer warps read their 16-byte units straight from
//    HBM (coalesced 16-byte loads, the next unit's loads issued before the
//    current unit is counted), convert and count.  Staging the frames in
//    shared memory instead (1-D bulk copies) was measured slower: the stages
//    take the room of four counting warps and their per-chunk handshake
//    costs more than the loads it hides (3.14 vs 3.41 TB/s on 1080p).
//  * The bin needs no clamp: with x = 16*(298Y + k_c) + offset, x >> 16 is an
//    "extended" bin covering every byte triple; extended bins outside [0,16)
//    fold into bins 0 and 15 when the table is flushed
//    (clamp(x >> 8, 0, 255) >> 4 == clamp(x >> 12, 0, 15)).
//  * Per pixel and channel: one dp2a (byte select, multiply, add the chroma
//    term and the table row base), one prmt (shared address = row byte(s) of
//    x + the lane's column byte) and one shared-memory reduction.  Each lane
//    owns a column ([row][lane], 256-byte rows); four warps share a table
//    region (two column halves x two 16-bit counter halves), so the reductions
//    never conflict on a bank and 20 warps fit in shared memory.
//  * After each item the table is flushed (lane columns and counter halves
//    summed, extended bins folded) into one of two accumulators and handed to a
//    publisher warp, which publishes it while the consumers go on counting:
//    directly to hist[k] when the item is the whole frame, else through a global
//    accumulator that the CTA completing the frame turns into hist[k].  The CTA completing the second
//    frame of a consecutive pair computes that pair's score.  Completion uses
//    counters; no CTA waits for another.
//  * Two kernels share all of the above.  hist_kernel: every item is counted
//    by all 20 consumer warps (one frame in flight per SM), each table region
//    flushing its own rows.  hist_kernel_rg (queue launches of frames up to
//    kRegionFramePxMax pixels): each 4-warp table region takes whole items of
//    its own, popped by its first thread one item ahead, so an item's flush
//    reads and zeroes one region's table instead of five - at 640 x 360 the
//    flushes of the first kernel are an eighth of its shared-memory traffic,
//    at 1080p 1.4 %, where five frames in flight per SM cost more than that.
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
static_assert(kRowsR + kRowsG + kRowsB == kTabRowsPerRegion, "table rows");

// x_c = 4768*Y + K_c, K_c = 16*(chroma term + 128 - 298*16 + off_c*4096) + (row base << 16)
// 4768 = 298*16; chroma weights *16: 409 -> 6544, 516 -> 8256, -100 -> -1600, -208 -> -3328.
constexpr uint32_t kWY = 4768u;
constexpr uint32_t kWV_R = 6544u;
constexpr uint32_t kWU_B = 8256u;
constexpr int32_t kWU_G = -1600, kWV_G = -3328;
constexpr int32_t kCR = 16 * (-409 * 128 + 128 - 298 * 16 + kOffR * 4096);             // 5632
constexpr int32_t kCB = 16 * (-516 * 128 + 128 - 298 * 16 + kOffB * 4096);             // 48640
constexpr int32_t kCG = 16 * (100 * 128 + 208 * 128 + 128 - 298 * 16 + kOffG * 4096);  // 1277440
static_assert(kCR == 5632 && kCB == 48640 && kCG == 1277440, "chroma constants");

constexpr int kNT = kConsumerThreads;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

// Description of one chunk (rows [r0, r0 + rows) of element k of job `job`),
// written by the producer before it arrives on the slot's barrier.  job < 0
// marks the end of the CTA's work.
struct ChunkMeta {
    int32_t job, k, rows, seg_end, seg_rp, r0, pad[2];
};

// What the publisher warp needs to publish one flushed item: its job, element
// and row pairs (job < 0: the consumers are done).
struct PubMeta {
    int32_t job, k, seg_rp, pad;
};

struct Smem {
    uint8_t* tab;
    ChunkMeta* meta;    // [kStages]
    uint32_t* acc;      // [2][64]: flushed counts of an item, double-buffered for the publisher
    PubMeta* pmeta;     // [2]
    uint64_t* full;     // [kStages]
    uint64_t* empty;    // [kStages]
    uint64_t* cbar;     // [kRegions] barrier of one table region's consumer warps
    uint64_t* accfull;  // [2] acc[b] holds an item's counts (each region's first thread arrives)
    uint64_t* accfree;  // [2] the publisher has taken acc[b] (its 32 lanes arrive)
    int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* smem) {
    Smem s;
    s.tab = smem;
    s.meta = reinterpret_cast<ChunkMeta*>(smem + kTabBytes);
    s.acc = reinterpret_cast<uint32_t*>(s.meta + kStages);
    s.pmeta = reinterpret_cast<PubMeta*>(s.acc + 128);
    s.full = reinterpret_cast<uint64_t*>(s.pmeta + 2);
    s.empty = s.full + kStages;
    s.cbar = s.empty + kStages;
    s.accfull = s.cbar + kRegions;
    s.accfree = s.accfull + 2;
    s.abort_flag = reinterpret_cast<int*>(s.accfree + 2);
    return s;
}
static_assert(kStages * sizeof(ChunkMeta) + 128 * 4 + 2 * sizeof(PubMeta) + (2 * kStages + kRegions + 4) * 8 + 16 <=
                  kSmemMisc,
              "misc smem");

struct SmemRg {
    uint8_t* tab;
    ChunkMeta* slot;    // [kRegions][2] the region's current and next chunk
    uint32_t* acc;      // [kRegions][2][64]: flushed counts of an item, double-buffered for the publisher
    PubMeta* pmeta;     // [kRegions][2]
    uint64_t* cbar;     // [kRegions] barrier of one table region's consumer warps
    uint64_t* accfull;  // [kRegions][2] acc holds an item's counts (the region's first thread arrives)
    uint64_t* accfree;  // [kRegions][2] the publisher has taken acc (its 32 lanes arrive)
    int* abort_flag;
};

__device__ __forceinline__ SmemRg carve_rg(uint8_t* smem) {
    SmemRg s;
    s.tab = smem;
    s.acc = reinterpret_cast<uint32_t*>(smem + kTabBytes);
    s.slot = reinterpret_cast<ChunkMeta*>(s.acc + kRegions * 2 * 64);
    s.pmeta = reinterpret_cast<PubMeta*>(s.slot + kRegions * 2);
    s.cbar = reinterpret_cast<uint64_t*>(s.pmeta + kRegions * 2);
    s.accfull = s.cbar + kRegions;
    s.accfree = s.accfull + kRegions * 2;
    s.abort_flag = reinterpret_cast<int*>(s.accfree + kRegions * 2);
    return s;
}
static_assert(kRegions * (2 * 64 * 4 + 2 * sizeof(ChunkMeta) + 2 * sizeof(PubMeta) + 5 * 8) + 16 <= kSmemMisc,
              "misc smem (region streams)");

__device__ __forceinline__ const Job& job_of(const Launch& L, int j) { return L.jobs ? L.jobs[j] : L.job0; }

// how long a bounded wait of this launch waits before it gives up
__device__ __forceinline__ uint64_t wait_limit(const Launch& L) {
    return L.wait_limit_ns ? L.wait_limit_ns : kWaitLimitNs;
}

// elements of job0 when its count lives on the device
__device__ __forceinline__ int64_t device_elems(const Launch& L) {
    return L.d_count ? static_cast<int64_t>(L.count_mul) * static_cast<int64_t>(*L.d_count) : L.job0.n;
}

template <class S>
__device__ __forceinline__ void fail(const Launch& L, const S& s) {
    *reinterpret_cast<volatile int*>(s.abort_flag) = 1;
    atomicOr(L.status, kStatusTimeout);
}

template <class S>
__device__ __forceinline__ bool aborted(const S& s) {
    return *reinterpret_cast<volatile int*>(s.abort_flag) != 0;
}

__device__ __forceinline__ Item item_at(const Launch& L, int64_t i) {
    if (L.items) return L.items[i];
    const Job& J = L.job0;
    Item it;
    it.job = 0;
    if (J.tail_parts > 0 && i >= J.tail_from) {
        const int64_t j = i - J.tail_from;
        it.k = static_cast<int32_t>(J.tail_from + j / J.tail_parts);
        it.rp0 = static_cast<int32_t>(j - (it.k - J.tail_from) * static_cast<int64_t>(J.tail_parts)) * J.tail_rp;
        it.nrp = min(J.tail_rp, J.H / 2 - it.rp0);
        return it;
    }
    it.k = static_cast<int32_t>(i / J.items_per_frame);
    const int part = static_cast<int>(i - static_cast<int64_t>(it.k) * J.items_per_frame);
    it.rp0 = part * J.item_rp;
    it.nrp = min(J.item_rp, J.H / 2 - it.rp0);
    return it;
}

// ---------------------------------------------------------------------------
// producer: one thread walks this CTA's work (popped items, or one contiguous
// range of row pairs) and hands out its chunk descriptors
// ---------------------------------------------------------------------------

// Hand out one chunk: rows [r, r + rows) of element k of job j.  Returns false
// when the wait for a free slot gave up.
__device__ __forceinline__ bool stage_chunk(const Launch& L, const Smem& s, uint32_t it, int j, int32_t k, int r,
                                            int rows, bool seg_end, int seg_rp) {
    const uint32_t st = it % kStages;
    if (it >= static_cast<uint32_t>(kStages)) {
        if (!ptx::mbar_wait_bounded(&s.empty[st], ((it / kStages) - 1) & 1u, wait_limit(L))) {
            fail(L, s);
            return false;
        }
    }
    ChunkMeta& m = s.meta[st];
    m.job = j;
    m.k = k;
    m.rows = rows;
    m.seg_end = seg_end;
    m.seg_rp = seg_rp;
    m.r0 = r;
    ptx::mbar_arrive(&s.full[st]);  // release: the descriptor is visible to the waiting consumers
    return true;
}

// Test hook: with withhold_after = k >= 0 the producer hands out k chunks and
// then nothing more (no end marker either), so the consumers' bounded waits run
// out and the launch ends with the timeout bit in the status word.
__device__ __forceinline__ bool withheld(const Launch& L, uint32_t it) {
    return L.withhold_after >= 0 && it >= static_cast<uint32_t>(L.withhold_after);
}

// ---------------------------------------------------------------------------
// work of a table region: each region's first thread walks its share of the
// CTA's work (popped items, or a contiguous range of row pairs) and hands its
// four warps one chunk at a time, so that a frame is counted (and its table
// flushed) by one region only
// ---------------------------------------------------------------------------
struct RegionSource {
    bool queue;              // items popped from the launch's queue (else a contiguous range)
    bool have_item, have_next, ended;
    Item item;
    uint64_t next;           // index of the next item, popped one item ahead
    int r, r_end;            // luma rows of the current item still to hand out
    int64_t g, g_end, k;     // contiguous mode: row pairs [g, g_end), current element k
    int rp, seg;             //   row pair within element k, row pairs of the open segment
    uint32_t handed;         // chunks handed out (test hook)
};

__device__ __forceinline__ int64_t queue_items(const Launch& L) {
    return L.d_count ? device_elems(L) * L.job0.items_per_frame : L.n_items;
}

__device__ void src_init(RegionSource& q, const Launch& L, int region) {
    q.handed = 0;
    q.have_item = q.have_next = q.ended = false;
    q.queue = L.rp_per_cta == 0;
    if (q.queue) return;
    // the CTA's contiguous range of job0's row pairs, split evenly over its regions;
    // segments end at frame edges and every item_rp row pairs (16-bit bound)
    const Job& J = L.job0;
    const int hp = J.H / 2;
    const int64_t total_rp = device_elems(L) * hp;
    const int64_t rpc = L.rp_per_cta > 0 ? L.rp_per_cta : (total_rp + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = min(static_cast<int64_t>(blockIdx.x) * rpc, total_rp);
    const int64_t c1 = min(c0 + rpc, total_rp);
    const int64_t per = (c1 - c0 + kRegions - 1) / kRegions;
    q.g = min(c0 + region * per, c1);
    q.g_end = min(q.g + per, c1);
    q.k = q.g / hp;
    q.rp = static_cast<int>(q.g - q.k * hp);
    q.seg = 0;
}

// pop one item index (the region that first finds the queue empty counts itself
// done; the last of all regions resets the queue, so a launch leaves it zero)
__device__ __forceinline__ uint64_t pop_item(RegionSource& q, const Launch& L) {
    const uint64_t i = atomicAdd(reinterpret_cast<unsigned long long*>(L.queue), 1ull);
    if (i >= static_cast<uint64_t>(queue_items(L)) && !q.ended) {
        q.ended = true;
        const uint32_t old = atomicAdd(&L.queue[2], 1u);
        if (old == gridDim.x * kRegions - 1) {
            atomicExch(reinterpret_cast<unsigned long long*>(L.queue), 0ull);
            atomicExch(&L.queue[2], 0u);
        }
    }
    return i;
}

// the region's next chunk (job < 0: no more)
__device__ ChunkMeta src_next(RegionSource& q, const Launch& L) {
    ChunkMeta m{};
    m.job = -1;
    if (!q.queue) {
        if (q.g >= q.g_end) return m;
        const Job& J = L.job0;
        const int hp = J.H / 2, crp = J.chunk_rows / 2, srp = J.item_rp;
        int mm = min(crp, hp - q.rp);
        if (q.g_end - q.g < mm) mm = static_cast<int>(q.g_end - q.g);
        mm = min(mm, srp - q.seg);
        const int nseg = q.seg + mm;
        const bool seg_end = (q.rp + mm == hp) || (q.g + mm == q.g_end) || (nseg == srp);
        m.job = 0;
        m.k = static_cast<int32_t>(q.k);
        m.rows = 2 * mm;
        m.seg_end = seg_end;
        m.seg_rp = nseg;
        m.r0 = 2 * q.rp;
        q.g += mm;
        q.rp += mm;
        q.seg = seg_end ? 0 : nseg;
        if (q.rp == hp) {
            q.rp = 0;
            ++q.k;
        }
        return m;
    }
    if (!q.have_item) {
        if (q.ended && !q.have_next) return m;
        const uint64_t i = q.have_next ? q.next : pop_item(q, L);
        q.have_next = false;
        if (i >= static_cast<uint64_t>(queue_items(L))) return m;
        q.item = item_at(L, static_cast<int64_t>(i));
        q.r = 2 * q.item.rp0;
        q.r_end = 2 * (q.item.rp0 + q.item.nrp);
        q.have_item = true;
        if (!q.ended) {  // the next item's index, one item ahead (its latency hides behind this item)
            q.next = pop_item(q, L);
            q.have_next = true;
        }
    }
    const Job& J = job_of(L, q.item.job);
    const int rows = min(J.chunk_rows, q.r_end - q.r);
    m.job = q.item.job;
    m.k = q.item.k;
    m.rows = rows;
    m.seg_end = q.r + rows == q.r_end;
    m.seg_rp = q.item.nrp;
    m.r0 = q.r;
    q.r += rows;
    if (m.seg_end) q.have_item = false;
    return m;
}

__device__ void produce(const Launch& L, const Smem& s) {
    uint32_t it = 0;
    bool stop = false;  // withheld (test hook)
    if (L.rp_per_cta != 0) {
        // Contiguous split of job0's row pairs: every CTA does the same work and
        // flushes only at frame edges or every item_rp row pairs (16-bit bound).
        const Job& J = L.job0;
        const int hp = J.H / 2, crp = J.chunk_rows / 2, srp = J.item_rp;
        const int64_t total_rp = device_elems(L) * hp;
        const int64_t rpc = L.rp_per_cta > 0 ? L.rp_per_cta : (total_rp + gridDim.x - 1) / gridDim.x;
        int64_t g = blockIdx.x * rpc;
        const int64_t g_end = min(g + rpc, total_rp);
        int64_t k = g / hp;
        int rp = static_cast<int>(g - k * hp);
        int seg = 0;
        while (g < g_end && !aborted(s)) {
            if (withheld(L, it)) {
                stop = true;
                break;
            }
            int m = min(crp, hp - rp);
            if (g_end - g < m) m = static_cast<int>(g_end - g);
            m = min(m, srp - seg);
            const int nseg = seg + m;
            const bool seg_end = (rp + m == hp) || (g + m == g_end) || (nseg == srp);
            if (!stage_chunk(L, s, it, 0, static_cast<int32_t>(k), 2 * rp, 2 * m, seg_end, nseg)) break;
            ++it;
            g += m;
            rp += m;
            seg = seg_end ? 0 : nseg;
            if (rp == hp) {
                rp = 0;
                ++k;
            }
        }
    } else {
        const int64_t n_items = L.d_count ? device_elems(L) * L.job0.items_per_frame : L.n_items;
        while (!aborted(s) && !stop) {
            const uint64_t i = atomicAdd(reinterpret_cast<unsigned long long*>(L.queue), 1ull);
            if (i >= static_cast<uint64_t>(n_items)) break;
            const Item item = item_at(L, static_cast<int64_t>(i));
            const Job& J = job_of(L, item.job);
            const int r_end = 2 * (item.rp0 + item.nrp);
            bool ok = true;
            for (int r = 2 * item.rp0; r < r_end && ok && !aborted(s); r += J.chunk_rows) {
                if (withheld(L, it)) {
                    stop = true;
                    break;
                }
                const int rows = min(J.chunk_rows, r_end - r);
                ok = stage_chunk(L, s, it, item.job, item.k, r, rows, r + rows == r_end, item.nrp);
                if (ok) ++it;
            }
        }
        // the last CTA done with the queue resets it (every other CTA has made
        // its last pop by then)
        const uint32_t old = atomicAdd(&L.queue[2], 1u);
        if (old == gridDim.x - 1) {
            atomicExch(reinterpret_cast<unsigned long long*>(L.queue), 0ull);
            atomicExch(&L.queue[2], 0u);
        }
    }
    // Tell the consumers: a descriptor with job = -1.
    if (!aborted(s) && !stop) {
        const uint32_t st = it % kStages;
        bool ok = true;
        if (it >= static_cast<uint32_t>(kStages)) {
            ok = ptx::mbar_wait_bounded(&s.empty[st], ((it / kStages) - 1) & 1u, wait_limit(L));
            if (!ok) fail(L, s);
        }
        if (ok) {
            s.meta[st].job = -1;
            ptx::mbar_arrive(&s.full[st]);
        }
    }
}

// ---------------------------------------------------------------------------
// consumers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_shared(uint32_t addr, uint32_t v) {
    // no memory clobber: the table is only read after the consumer barrier (whose
    // arrive and wait have one)
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// d.b0 = lane column byte, d.b1/d.b2 = bytes 2/3 of x (the table row), d.b3 = 0
__device__ __forceinline__ uint32_t tab_addr(uint32_t x, uint32_t lanereg) { return ptx::prmt(x, lanereg, 0x5324u); }

__device__ __forceinline__ void count3(uint32_t lanereg, uint32_t inc, uint32_t xr, uint32_t xg, uint32_t xb) {
    red_shared(tab_addr(xr, lanereg), inc);
    red_shared(tab_addr(xg, lanereg), inc);
    red_shared(tab_addr(xb, lanereg), inc);
}

// 32 pixels: 16 columns of two luma rows sharing 8 chroma samples.
__device__ __forceinline__ void count_unit(uint32_t lanereg, uint32_t inc, uint32_t cR, uint32_t cG, uint32_t cB,
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
        // chroma sample in bytes 0,1 serves luma bytes 0,1; bytes 2,3 serve luma bytes 2,3
        {
            const uint32_t kr = ptx::dp2a_lo_uu(aR, uvw[w], cR);
            const uint32_t kb = ptx::dp2a_lo_uu(aB, uvw[w], cB);
            const uint32_t kg = static_cast<uint32_t>(ptx::dp2a_lo_su(aG, uvw[w], static_cast<int32_t>(cG)));
            count3(lanereg, inc, ptx::dp2a_lo_uu(aY0, yw0[w], kr), ptx::dp2a_lo_uu(aY0, yw0[w], kg),
                   ptx::dp2a_lo_uu(aY0, yw0[w], kb));
            count3(lanereg, inc, ptx::dp2a_lo_uu(aY1, yw0[w], kr), ptx::dp2a_lo_uu(aY1, yw0[w], kg),
                   ptx::dp2a_lo_uu(aY1, yw0[w], kb));
            count3(lanereg, inc, ptx::dp2a_lo_uu(aY0, yw1[w], kr), ptx::dp2a_lo_uu(aY0, yw1[w], kg),
                   ptx::dp2a_lo_uu(aY0, yw1[w], kb));
            count3(lanereg, inc, ptx::dp2a_lo_uu(aY1, yw1[w], kr), ptx::dp2a_lo_uu(aY1, yw1[w], kg),
                   ptx::dp2a_lo_uu(aY1, yw1[w], kb));
        }
        {
            const uint32_t kr = ptx::dp2a_hi_uu(aR, uvw[w], cR);
            const uint32_t kb = ptx::dp2a_hi_uu(aB, uvw[w], cB);
            const uint32_t kg = static_cast<uint32_t>(ptx::dp2a_hi_su(aG, uvw[w], static_cast<int32_t>(cG)));
            count3(lanereg, inc, ptx::dp2a_hi_uu(aY0, yw0[w], kr), ptx::dp2a_hi_uu(aY0, yw0[w], kg),
                   ptx::dp2a_hi_uu(aY0, yw0[w], kb));
            count3(lanereg, inc, ptx::dp2a_hi_uu(aY1, yw0[w], kr), ptx::dp2a_hi_uu(aY1, yw0[w], kg),
                   ptx::dp2a_hi_uu(aY1, yw0[w], kb));
            count3(lanereg, inc, ptx::dp2a_hi_uu(aY0, yw1[w], kr), ptx::dp2a_hi_uu(aY0, yw1[w], kg),
                   ptx::dp2a_hi_uu(aY0, yw1[w], kb));
            count3(lanereg, inc, ptx::dp2a_hi_uu(aY1, yw1[w], kr), ptx::dp2a_hi_uu(aY1, yw1[w], kg),
                   ptx::dp2a_hi_uu(aY1, yw1[w], kb));
        }
    }
}

// Flush of one table region by its own consumer threads (rt = thread within
// the region): every row summed over its 64 words and both 16-bit halves,
// extended bin folded into the final bin, added into acc[48]; the region's
// rows are left zeroed.
__device__ __forceinline__ void flush_region(uint8_t* tab, uint32_t* acc, int region, int rt) {
    const int lane = rt & 31;
    for (int row = region * kTabRowsPerRegion + rt; row < (region + 1) * kTabRowsPerRegion; row += kRegionThreads) {
        uint8_t* p = tab + row * 256;
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            uint4* q = reinterpret_cast<uint4*>(p + ((lane + i) & 15) * 16);
            const uint4 v = *q;
            lo += (v.x & 0xFFFFu) + (v.y & 0xFFFFu) + (v.z & 0xFFFFu) + (v.w & 0xFFFFu);
            hi += (v.x >> 16) + (v.y >> 16) + (v.z >> 16) + (v.w >> 16);
            *q = make_uint4(0, 0, 0, 0);
        }
        const uint32_t sum = lo + hi;
        const int t = row % kTabRowsPerRegion;
        int c, e, off;
        if (t < kBaseG) { c = 0; e = t - kBaseR; off = kOffR; }
        else if (t < kBaseB) { c = 1; e = t - kBaseG; off = kOffG; }
        else { c = 2; e = t - kBaseB; off = kOffB; }
        const int b = min(max(e - off, 0), 15);
        if (sum) atomicAdd(&acc[c * 16 + b], sum);
    }
}

// Score of element k from two histograms (h0, p0: bins lane; h1, p1: bins 32 + lane).
__device__ __forceinline__ void write_score(const Job& J, int64_t k, uint32_t h0, uint32_t h1, uint32_t p0, uint32_t p1,
                                            int lane) {
    uint32_t d = (h0 > p0 ? h0 - p0 : p0 - h0);
    if (lane < 16) d += (h1 > p1 ? h1 - p1 : p1 - h1);
    const uint32_t s = __reduce_add_sync(0xffffffffu, d);
    if (lane == 0) {
        // a gated pass (score_at set) writes the score of its pair (2i, 2i+1) to element score_at[i]
        const int64_t o = J.score_at ? J.score_at[k >> 1] : k;
        J.score[o] = s;
        J.flag[o] = (2ull * s > static_cast<uint64_t>(J.W) * J.H) ? 1 : 0;
    }
}

// The publisher warp: publish an item's counts of element k (seg_rp row pairs;
// lane holds bins lane and 32 + lane), complete the frame and the scores it
// unblocks.
__device__ void publish(const Job& J, int64_t n, int64_t k, int seg_rp, uint32_t h0, uint32_t h1, int lane) {
    const int hp = J.H / 2;
    if (seg_rp != hp) {
        // part of the frame: accumulate; the CTA completing the frame finishes it
        uint32_t* pk = J.partial + k * 48;
        if (h0) atomicAdd(pk + lane, h0);
        if (lane < 16 && h1) atomicAdd(pk + 32 + lane, h1);
        __threadfence();
        __syncwarp();
        uint32_t old = 0;
        if (lane == 0) old = atomicAdd(&J.done[k], static_cast<uint32_t>(seg_rp));
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old + static_cast<uint32_t>(seg_rp) != static_cast<uint32_t>(hp)) return;
        __threadfence();
        h0 = ptx::ld_cg_u32(pk + lane);
        h1 = lane < 16 ? ptx::ld_cg_u32(pk + 32 + lane) : 0u;
        pk[lane] = 0;  // leave the accumulator zeroed for the next call
        if (lane < 16) pk[32 + lane] = 0;
        if (lane == 0) J.done[k] = 0;
    }
    J.hist[k * 48 + lane] = h0;
    if (lane < 16) J.hist[k * 48 + 32 + lane] = h1;
    if (!J.score) return;
    __threadfence();
    __syncwarp();
    // a gated pass needs only the scores of its pairs (2i, 2i+1): the odd elements
    const bool want0 = k > 0 && (!J.score_at || (k & 1));
    const bool want1 = k + 1 < n && (!J.score_at || !(k & 1));
    if (k == 0 && lane == 0 && !J.score_at) {
        J.score[0] = 0;
        J.flag[0] = 0;
    }
    // both stencil pairs of element k at once, (k - 1, k) counted by lane 0 and (k, k + 1) by
    // lane 1: the second arrival of a pair computes its score
    uint32_t old = 0;
    if (lane == 0 && want0) old = atomicAdd(&J.pair[k], 1u);
    if (lane == 1 && want1) old = atomicAdd(&J.pair[k + 1], 1u);
    const bool s0 = __shfl_sync(0xffffffffu, old, 0) == 1u;
    const bool s1 = __shfl_sync(0xffffffffu, old, 1) == 1u;
    if (!s0 && !s1) return;
    __threadfence();
    // the neighbours' histograms, every load in flight together
    uint32_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    if (s0) {
        a0 = ptx::ld_cg_u32(J.hist + (k - 1) * 48 + lane);
        if (lane < 16) a1 = ptx::ld_cg_u32(J.hist + (k - 1) * 48 + 32 + lane);
    }
    if (s1) {
        b0 = ptx::ld_cg_u32(J.hist + (k + 1) * 48 + lane);
        if (lane < 16) b1 = ptx::ld_cg_u32(J.hist + (k + 1) * 48 + 32 + lane);
    }
    if (s0) {
        write_score(J, k, h0, h1, a0, a1, lane);
        if (lane == 0) J.pair[k] = 0;
    }
    if (s1) {
        write_score(J, k + 1, h0, h1, b0, b1, lane);
        if (lane == 0) J.pair[k + 1] = 0;
    }
}

__device__ __forceinline__ uint4 ldg128(const uint8_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

// Barrier of one table region's consumer threads, bounded: every one of them
// arrives (release) and waits (acquire) for the phase.  A consumer that gave up
// earlier has left the loop, so the others would wait for it forever on a named
// barrier; here they give up too, after the launch's wait limit.
__device__ __forceinline__ bool consumer_sync(const Launch& L, const Smem& s, int region, uint32_t& phase) {
    ptx::mbar_arrive(&s.cbar[region]);
    const bool ok = ptx::mbar_wait_bounded(&s.cbar[region], phase & 1u, wait_limit(L));
    ++phase;
    if (!ok) fail(L, s);
    return ok;
}


__device__ void consume(const Launch& L, const Smem& s, int warp, int lane) {
    const int ctid = warp * 32 + lane;
    const int region = warp / kGroupWarps;
    const int rt = ctid - region * kRegionThreads;  // thread within the region
    const uint32_t lanereg = static_cast<uint32_t>(lane * 4 + (warp & 1) * 128);
    const uint32_t inc = (warp & 2) ? 65536u : 1u;
    // table row of x = (x >> 16): shared base / 256 + region rows + channel rows + extended bin
    const uint32_t rowbase = ((ptx::smem_u32(s.tab) >> 8) + static_cast<uint32_t>(region * kTabRowsPerRegion)) << 16;
    const uint32_t cR = static_cast<uint32_t>(kCR) + rowbase + (static_cast<uint32_t>(kBaseR) << 16);
    const uint32_t cG = static_cast<uint32_t>(kCG) + rowbase + (static_cast<uint32_t>(kBaseG) << 16);
    const uint32_t cB = static_cast<uint32_t>(kCB) + rowbase + (static_cast<uint32_t>(kBaseB) << 16);
    uint32_t it = 0;
    uint32_t cphase = 0;  // completed phases of the consumer barrier
    uint32_t seg = 0;     // items flushed so far (acc buffer seg & 1)
    int rot = 0;
    // geometry of the current job, kept in registers: reloaded only when a chunk
    // belongs to another job (global loads at every chunk start stall all warps)
    int cur_job = -1, W = 0, H = 0, wv = 1, sc = 0;
    uint32_t dY = 0, dU = 0;
    float inv_wv = 1.f;
    for (;; ++it) {
        const uint32_t st = it % kStages;
        // Every consumer reaches the same chunk before any of them gives up, so
        // they leave the loop together (no named barrier is left half-full).
        if (aborted(s)) break;
        if (!ptx::mbar_wait_bounded(&s.full[st], (it / kStages) & 1u, wait_limit(L))) {
            fail(L, s);
            break;
        }
        const ChunkMeta m = s.meta[st];
        if (m.job < 0) break;
        const Job& J = job_of(L, m.job);
        if (m.job != cur_job) {
            cur_job = m.job;
            W = J.W;
            wv = J.wv;
            sc = J.sc;
            H = J.H;
            dY = J.dY;
            dU = J.dU;
            inv_wv = J.inv_wv;
        }
        const uint8_t* frame = J.nv12 + static_cast<int64_t>(J.slot[m.k]) * J.stride;
        const int units = (m.rows / 2) * wv;
        int u = ctid - rot;
        if (u < 0) u += kNT;
        const int p0 = static_cast<int>((static_cast<float>(u) + 0.5f) * inv_wv);
        int c = u - p0 * wv;
        // unit u of the chunk: row pair p0 + (u / wv), 16-byte column c; luma rows
        // r0 + 2p, r0 + 2p + 1 and chroma row r0/2 + p
        const uint8_t* ya = frame + static_cast<int64_t>(m.r0 + 2 * p0) * W + c * 16;
        const uint8_t* ua = frame + static_cast<int64_t>(W) * H + static_cast<int64_t>(m.r0 / 2 + p0) * W + c * 16;
        uint4 y0{}, y1{}, uv{};
        if (u < units) {
            y0 = ldg128(ya);
            y1 = ldg128(ya + W);
            uv = ldg128(ua);
        }
        for (; u < units; u += kNT) {
            // next unit: kNT units on; a column wrap adds one more row pair and
            // removes a row of columns (luma +2W-W, chroma +W-W).  Its loads are
            // issued before this unit is counted.
            ya += dY;
            ua += dU;
            c += sc;
            if (c >= wv) {
                c -= wv;
                ya += W;
            }
            uint4 ny0{}, ny1{}, nuv{};
            if (u + kNT < units) {
                ny0 = ldg128(ya);
                ny1 = ldg128(ya + W);
                nuv = ldg128(ua);
            }
            count_unit(lanereg, inc, cR, cG, cB, y0, y1, uv);
            y0 = ny0;
            y1 = ny1;
            uv = nuv;
        }
        rot = (rot + units) % kNT;
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&s.empty[st]);
        if (m.seg_end) {
            // each table region flushes on its own as soon as its four warps have counted
            // the item; the other regions may still be counting it or already be on the next
            const uint32_t b = seg & 1u;
            if (!consumer_sync(L, s, region, cphase)) break;  // the region has counted the item
            // acc[b] was last filled two items ago: the publisher has taken it
            if (seg >= 2 && !ptx::mbar_wait_bounded(&s.accfree[b], ((seg >> 1) - 1) & 1u, wait_limit(L))) {
                fail(L, s);
                break;
            }
            flush_region(s.tab, s.acc + 64 * b, region, rt);
            if (!consumer_sync(L, s, region, cphase)) break;  // region rows zeroed, its part of acc[b] added
            if (rt == 0) {
                if (region == 0) s.pmeta[b] = PubMeta{m.job, m.k, m.seg_rp, 0};
                ptx::mbar_arrive(&s.accfull[b]);  // release; the phase completes with the last region
            }
            ++seg;
        }
    }
    // tell the publisher that no item follows (not after a failure: it then gives up by itself)
    if (!aborted(s) && rt == 0) {
        const uint32_t b = seg & 1u;
        if (seg < 2 || ptx::mbar_wait_bounded(&s.accfree[b], ((seg >> 1) - 1) & 1u, wait_limit(L))) {
            if (region == 0) s.pmeta[b] = PubMeta{-1, 0, 0, 0};
            ptx::mbar_arrive(&s.accfull[b]);
        } else {
            fail(L, s);
        }
    }
}

// The publisher warp: takes each flushed item's counts off acc[b] (freeing the
// buffer for the consumers at once) and publishes them - global atomics, frame
// completion, the score of each completed pair - so that the latency of those
// global round trips is not on the consumers' path.
__device__ void publisher(const Launch& L, const Smem& s, int lane) {
    const int64_t n_dev = device_elems(L);
    for (uint32_t pseg = 0;; ++pseg) {
        const uint32_t b = pseg & 1u;
        if (!ptx::mbar_wait_bounded(&s.accfull[b], (pseg >> 1) & 1u, wait_limit(L))) {
            fail(L, s);
            return;
        }
        const PubMeta pm = s.pmeta[b];
        if (pm.job < 0) return;
        uint32_t* acc = s.acc + 64 * b;
        const uint32_t h0 = acc[lane];
        const uint32_t h1 = lane < 16 ? acc[32 + lane] : 0u;
        acc[lane] = 0;
        if (lane < 16) acc[32 + lane] = 0;
        ptx::mbar_arrive(&s.accfree[b]);  // release: acc[b] read and zeroed
        const Job& J = job_of(L, pm.job);
        publish(J, L.d_count ? n_dev : J.n, pm.k, pm.seg_rp, h0, h1, lane);
    }
}

__global__ void __launch_bounds__(kHistThreads, 1) hist_kernel(const __grid_constant__ Launch L) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const Smem s = carve(smem);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kTabBytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid < 128) s.acc[tid] = 0;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&s.full[i], 1);
            ptx::mbar_init(&s.empty[i], kConsumerWarps);
        }
        for (int r = 0; r < kRegions; ++r) ptx::mbar_init(&s.cbar[r], kRegionThreads);
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.accfull[i], kRegions);
            ptx::mbar_init(&s.accfree[i], 32);
        }
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    // the table is zeroed and the barriers set up while the previous kernel in the
    // stream may still be finishing; global memory only after it has completed
    ptx::pdl_wait();
    ptx::pdl_release();
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0) produce(L, s);
        return;
    }
    if (warp == kConsumerWarps + 1) {
        publisher(L, s, lane);
        return;
    }
    consume(L, s, warp, lane);
}

// Barrier of one table region's consumer threads, bounded: every one of them
// arrives (release) and waits (acquire) for the phase.  A consumer that gave up
// earlier has left the loop, so the others would wait for it forever on a named
// barrier; here they give up too, after the launch's wait limit.
__device__ __forceinline__ bool consumer_sync_rg(const Launch& L, const SmemRg& s, int region, uint32_t& phase) {
    ptx::mbar_arrive(&s.cbar[region]);
    const bool ok = ptx::mbar_wait_bounded(&s.cbar[region], phase & 1u, wait_limit(L));
    ++phase;
    if (!ok) fail(L, s);
    return ok;
}

// One table region (four warps): its first thread hands out the region's chunks
// through slot[region][2] (chunk c + 1 written while chunk c is counted, made
// visible by the region barrier that ends chunk c); all 128 threads count each
// chunk's units; at the end of an item the region flushes its table into one of
// its two accumulators and hands it to the publisher warp.
__device__ void consume_rg(const Launch& L, const SmemRg& s, int warp, int lane) {
    const int region = warp / kGroupWarps;
    const int rt = (warp - region * kGroupWarps) * 32 + lane;  // thread within the region
    const bool leader = rt == 0;
    ChunkMeta* slot = s.slot + 2 * region;
    uint32_t* racc = s.acc + region * 2 * 64;
    const uint32_t lanereg = static_cast<uint32_t>(lane * 4 + (warp & 1) * 128);
    const uint32_t inc = (warp & 2) ? 65536u : 1u;
    // table row of x = (x >> 16): shared base / 256 + region rows + channel rows + extended bin
    const uint32_t rowbase = ((ptx::smem_u32(s.tab) >> 8) + static_cast<uint32_t>(region * kTabRowsPerRegion)) << 16;
    const uint32_t cR = static_cast<uint32_t>(kCR) + rowbase + (static_cast<uint32_t>(kBaseR) << 16);
    const uint32_t cG = static_cast<uint32_t>(kCG) + rowbase + (static_cast<uint32_t>(kBaseG) << 16);
    const uint32_t cB = static_cast<uint32_t>(kCB) + rowbase + (static_cast<uint32_t>(kBaseB) << 16);
    RegionSource src;
    bool stop = false;  // the leader withholds the rest (test hook)
    if (leader) {
        src_init(src, L, region);
        if (withheld(L, 0)) {
            slot[0].job = -2;  // the region's warps stop; no end marker, so the publisher gives up
            stop = true;
        } else {
            slot[0] = src_next(src, L);
            src.handed = 1;
        }
    }
    uint32_t cphase = 0;  // completed phases of the region barrier
    uint32_t seg = 0;     // items flushed so far (acc buffer seg & 1)
    uint32_t par = 0;     // slot of the current chunk
    int rot = 0;
    // geometry of the current job, kept in registers: reloaded only when a chunk
    // belongs to another job (global loads at every chunk start stall all warps)
    int cur_job = -1, W = 0, H = 0, wv = 1, sc = 0;
    uint32_t dY = 0, dU = 0;
    float inv_wv = 1.f;
    if (!consumer_sync_rg(L, s, region, cphase)) return;  // slot[0] written
    for (;;) {
        if (aborted(s)) break;
        const ChunkMeta m = slot[par];
        if (m.job < 0) break;
        // the next chunk, while this one is counted (its slot was last read before the
        // barrier that started this chunk)
        if (leader) {
            if (withheld(L, src.handed)) {
                slot[par ^ 1u].job = -2;  // as above
                stop = true;
            } else {
                slot[par ^ 1u] = src_next(src, L);
                ++src.handed;
            }
        }
        const Job& J = job_of(L, m.job);
        if (m.job != cur_job) {
            cur_job = m.job;
            W = J.W;
            wv = J.wv;
            sc = J.sc_r;
            H = J.H;
            dY = J.dY_r;
            dU = J.dU_r;
            inv_wv = J.inv_wv;
        }
        const uint8_t* frame = J.nv12 + static_cast<int64_t>(J.slot[m.k]) * J.stride;
        const int units = (m.rows / 2) * wv;
        int u = rt - rot;
        if (u < 0) u += kRegionThreads;
        const int p0 = static_cast<int>((static_cast<float>(u) + 0.5f) * inv_wv);
        int c = u - p0 * wv;
        // unit u of the chunk: row pair p0 + (u / wv), 16-byte column c; luma rows
        // r0 + 2p, r0 + 2p + 1 and chroma row r0/2 + p
        const uint8_t* ya = frame + static_cast<int64_t>(m.r0 + 2 * p0) * W + c * 16;
        const uint8_t* ua = frame + static_cast<int64_t>(W) * H + static_cast<int64_t>(m.r0 / 2 + p0) * W + c * 16;
        uint4 y0{}, y1{}, uv{};
        if (u < units) {
            y0 = ldg128(ya);
            y1 = ldg128(ya + W);
            uv = ldg128(ua);
        }
        for (; u < units; u += kRegionThreads) {
            // next unit: kRegionThreads units on; a column wrap adds one more row pair
            // and removes a row of columns (luma +2W-W, chroma +W-W).  Its loads are
            // issued before this unit is counted.
            ya += dY;
            ua += dU;
            c += sc;
            if (c >= wv) {
                c -= wv;
                ya += W;
            }
            uint4 ny0{}, ny1{}, nuv{};
            if (u + kRegionThreads < units) {
                ny0 = ldg128(ya);
                ny1 = ldg128(ya + W);
                nuv = ldg128(ua);
            }
            count_unit(lanereg, inc, cR, cG, cB, y0, y1, uv);
            y0 = ny0;
            y1 = ny1;
            uv = nuv;
        }
        rot = (rot + units) % kRegionThreads;
        if (m.seg_end) {
            const uint32_t b = seg & 1u;
            if (!consumer_sync_rg(L, s, region, cphase)) break;  // the region has counted the item
            // acc[b] was last filled two items ago: the publisher has taken it
            if (seg >= 2 && !ptx::mbar_wait_bounded(&s.accfree[2 * region + b], ((seg >> 1) - 1) & 1u,
                                                    wait_limit(L))) {
                fail(L, s);
                break;
            }
            flush_region(s.tab, racc + 64 * b, region, rt);
            // rows zeroed, acc[b] complete, the next chunk's slot written
            if (!consumer_sync_rg(L, s, region, cphase)) break;
            if (leader) {
                s.pmeta[2 * region + b] = PubMeta{m.job, m.k, m.seg_rp, 0};
                ptx::mbar_arrive(&s.accfull[2 * region + b]);  // release: the counts and their item
            }
            ++seg;
        } else {
            if (!consumer_sync_rg(L, s, region, cphase)) break;  // the next chunk's slot written
        }
        par ^= 1u;
    }
    // tell the publisher that the region is done (not after a failure or a withheld
    // chunk: the publisher then gives up by itself)
    if (leader && !stop && !aborted(s)) {
        const uint32_t b = seg & 1u;
        if (seg < 2 || ptx::mbar_wait_bounded(&s.accfree[2 * region + b], ((seg >> 1) - 1) & 1u, wait_limit(L))) {
            s.pmeta[2 * region + b] = PubMeta{-1, 0, 0, 0};
            ptx::mbar_arrive(&s.accfull[2 * region + b]);
        } else {
            fail(L, s);
        }
    }
}

// The publisher warp: takes each flushed item's counts off a region's accumulator
// (freeing it for the region at once) and publishes them - global atomics, frame
// completion, the score of each completed pair - so that the latency of those
// global round trips is not on the consumers' path.  It polls the regions in turn
// and gives up when none has handed over an item for the launch's wait limit.
__device__ void publisher_rg(const Launch& L, const SmemRg& s, int lane) {
    const int64_t n_dev = device_elems(L);
    uint32_t pseg[kRegions];
    uint32_t live = (1u << kRegions) - 1u;  // regions not yet done
#pragma unroll
    for (int r = 0; r < kRegions; ++r) pseg[r] = 0;
    uint64_t t_last = ptx::globaltimer();
    uint32_t polls = 0;
    while (live) {
        bool any = false;
#pragma unroll
        for (int r = 0; r < kRegions; ++r) {
            if (!((live >> r) & 1u)) continue;
            const uint32_t b = pseg[r] & 1u;
            if (!ptx::mbar_try_wait(&s.accfull[2 * r + b], (pseg[r] >> 1) & 1u)) continue;
            any = true;
            const PubMeta pm = s.pmeta[2 * r + b];
            if (pm.job < 0) {
                live &= ~(1u << r);
                continue;
            }
            uint32_t* acc = s.acc + (2 * r + b) * 64;
            const uint32_t h0 = acc[lane];
            const uint32_t h1 = lane < 16 ? acc[32 + lane] : 0u;
            acc[lane] = 0;
            if (lane < 16) acc[32 + lane] = 0;
            ptx::mbar_arrive(&s.accfree[2 * r + b]);  // release: acc read and zeroed
            const Job& J = job_of(L, pm.job);
            publish(J, L.d_count ? n_dev : J.n, pm.k, pm.seg_rp, h0, h1, lane);
            ++pseg[r];
        }
        if (any) {
            t_last = ptx::globaltimer();
        } else {
            // nothing handed over: back off, the polls would take shared-memory cycles from
            // the counting (items take microseconds; each region has two accumulators)
            __nanosleep(256);
            if ((++polls & 15u) == 0 && ptx::globaltimer() - t_last > wait_limit(L)) {
                fail(L, s);
                return;
            }
        }
    }
}

__global__ void __launch_bounds__(kHistThreadsRg, 1) hist_kernel_rg(const __grid_constant__ Launch L) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const SmemRg s = carve_rg(smem);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kTabBytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < kRegions * 2 * 64; i += blockDim.x) s.acc[i] = 0;
    if (tid == 0) {
        for (int r = 0; r < kRegions; ++r) {
            ptx::mbar_init(&s.cbar[r], kRegionThreads);
            for (int i = 0; i < 2; ++i) {
                ptx::mbar_init(&s.accfull[2 * r + i], 1);
                ptx::mbar_init(&s.accfree[2 * r + i], 32);
            }
        }
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    ptx::pdl_wait();
    ptx::pdl_release();
    __syncthreads();
    if (warp == kConsumerWarps) {
        publisher_rg(L, s, lane);
        return;
    }
    consume_rg(L, s, warp, lane);
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

std::atomic<uint64_t> g_attr_done{0};  // kernel attribute set, one bit per device

}  // namespace

int chunk_rows_for(int W, int H, int requested) {
    (void)W;
    return (requested <= 0 || requested > H) ? H : requested;
}

void fill_job_consts(Job& j) {
    j.wv = j.W / 16;
    j.sp = kNT / j.wv;
    j.sc = kNT % j.wv;
    j.dY = static_cast<uint32_t>(j.sp * 2 * j.W + j.sc * 16);
    j.dU = static_cast<uint32_t>(j.sp * j.W + j.sc * 16);
    // the same steps for one table region's threads (the region-stream kernel)
    const int sp_r = kRegionThreads / j.wv;
    j.sc_r = kRegionThreads % j.wv;
    j.dY_r = static_cast<uint32_t>(sp_r * 2 * j.W + j.sc_r * 16);
    j.dU_r = static_cast<uint32_t>(sp_r * j.W + j.sc_r * 16);
    j.inv_wv = 1.0f / static_cast<float>(j.wv);
}

void choose_items(Job& j, int64_t item_px, int grid) {
    const int hp = j.H / 2;
    const int64_t frame_px = static_cast<int64_t>(j.W) * j.H;
    int64_t ipf;
    if (item_px > 0) {
        ipf = (frame_px + item_px - 1) / item_px;
    } else {
        // whole frames when there are plenty of them; else split frames so the
        // queue holds about 8 items per CTA
        const int64_t want = 8LL * grid * (region_frames(j.W, j.H) ? kRegions : 1);
        const int64_t n = std::max<int64_t>(j.n, 1);
        ipf = n >= want ? 1 : (want + n - 1) / n;
    }
    // an item stays under the 16-bit counter bound and holds at least one chunk
    const int64_t min_ipf = (frame_px + kItemPixelsMax - 1) / kItemPixelsMax;
    const int64_t max_ipf = std::max(1, hp / std::max(1, j.chunk_rows / 2));
    ipf = std::max(min_ipf, std::min(ipf, max_ipf));
    ipf = std::max<int64_t>(1, std::min<int64_t>(ipf, hp));
    j.item_rp = static_cast<int32_t>((hp + ipf - 1) / ipf);
    j.items_per_frame = (hp + j.item_rp - 1) / j.item_rp;
}

scn_status prepare_hist() {
    return once_per_device(g_attr_done, [] {
        SCN_CUDA_TRY(cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        SCN_CUDA_TRY(cudaFuncSetAttribute(hist_kernel_rg, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        return SCN_OK;
    });
}

scn_status launch_hist(const Launch& L, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(kTabBytes) + kSmemMisc;
    if (smem > static_cast<size_t>(kSmemLimit)) return SCN_EUNSUPPORTED;
    if (L.n_items <= 0 || L.grid <= 0) return SCN_OK;
    const scn_status sp = prepare_hist();
    if (sp != SCN_OK) return sp;
    if (L.region_items)
        SCN_CUDA_TRY(launch_pdl(hist_kernel_rg, dim3(L.grid), dim3(kHistThreadsRg), smem, st, L));
    else
        SCN_CUDA_TRY(launch_pdl(hist_kernel, dim3(L.grid), dim3(kHistThreads), smem, st, L));
    return SCN_OK;
}

HistShape resolve_hist_shape(const scn_seq* s) {
    HistShape sh;
    const int W = s->table->W, H = s->table->H;
    int sms = device_sm_count();
    if (sms <= 0) sms = 148;
    Job j{};
    j.W = W;
    j.H = H;
    j.n = std::max<int64_t>(s->n, 1);
    j.chunk_rows = chunk_rows_for(W, H, s->tune.chunk_rows);
    const int grid = s->tune.grid > 0 ? s->tune.grid : sms;
    choose_items(j, static_cast<int64_t>(s->tune.item_kpx) * 1000, grid);
    sh.chunk_rows = j.chunk_rows;
    sh.item_rp = j.item_rp;
    sh.items_per_frame = j.items_per_frame;
    const int64_t items = j.n * j.items_per_frame;
    sh.grid = static_cast<int>(std::min<int64_t>(grid, items));
    sh.rp_per_cta = 0;
    if (s->tune.item_kpx == 0 && j.n < 8LL * grid) {
        // no item size asked for and too few frames for whole-frame queue items:
        // one contiguous range of row pairs per CTA (perfect balance), flushed at
        // frame edges and at most every kItemPixelsMax pixels
        const int64_t total_rp = j.n * (H / 2);
        const int g = static_cast<int>(std::min<int64_t>(grid, total_rp));
        sh.rp_per_cta = (total_rp + g - 1) / g;
        sh.grid = static_cast<int>((total_rp + sh.rp_per_cta - 1) / sh.rp_per_cta);
        sh.item_rp = static_cast<int>(std::min<int64_t>(H / 2, std::max<int64_t>(1, kItemPixelsMax / (2LL * W))));
    }
    sh.smem = static_cast<size_t>(kTabBytes) + kSmemMisc;
    return sh;
}

// A single-sequence launch description (outputs and scratch filled in by the caller).
Launch single_launch(const scn_table* t, int64_t n, const int32_t* slot, const HistShape& sh) {
    Launch L{};
    Job& j = L.job0;
    j.nv12 = t->d_nv12;
    j.stride = t->frame_stride;
    j.slot = slot;
    j.n = n;
    j.W = t->W;
    j.H = t->H;
    j.chunk_rows = sh.chunk_rows;
    j.item_rp = sh.item_rp;
    j.items_per_frame = sh.items_per_frame;
    fill_job_consts(j);
    L.jobs = nullptr;
    L.items = nullptr;
    L.n_items = n * sh.items_per_frame;
    L.rp_per_cta = sh.rp_per_cta;
    L.grid = sh.grid;
    L.region_items = (sh.rp_per_cta == 0 && region_frames(t->W, t->H)) ? 1 : 0;
    // A queue of whole frames ends with every CTA on its last frame, finishing up to a frame's
    // time apart: the last `grid` frames are queued in kTailParts parts each instead, so the
    // launch ends on parts of frames.
    if (sh.rp_per_cta == 0 && !L.region_items && sh.items_per_frame == 1 && n >= 2LL * sh.grid &&
        n <= 0x7fffffff) {
        const int hp = t->H / 2;
        const int rp = (hp + kTailParts - 1) / kTailParts;
        j.tail_parts = (hp + rp - 1) / rp;
        if (j.tail_parts > 1) {
            j.tail_rp = rp;
            j.tail_from = static_cast<int32_t>(n - sh.grid);
            L.n_items = j.tail_from + static_cast<int64_t>(sh.grid) * j.tail_parts;
        } else {
            j.tail_parts = 0;
        }
    }
    return L;
}

static scn_status run_hist(scn_seq* s, uint32_t* d_hist, uint32_t* d_score, uint8_t* d_flag, void* stream) {
    if (!s || !d_hist) return SCN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_hist) & 3u) || (d_score && (reinterpret_cast<uintptr_t>(d_score) & 3u)))
        return SCN_EINVAL;
    if (s->n == 0) return SCN_OK;
    const HistShape sh = resolve_hist_shape(s);
    Launch L = single_launch(s->table, s->n, s->d_slot, sh);
    L.job0.hist = d_hist;
    L.job0.score = d_score;
    L.job0.flag = d_flag;
    L.job0.partial = s->d_partial;
    L.job0.done = s->d_done;
    L.job0.pair = s->d_pair;
    L.queue = s->d_queue;
    L.status = s->d_status;
    L.wait_limit_ns = s->test_wait_ns;
    L.withhold_after = s->test_withhold;
    return launch_hist(L, static_cast<cudaStream_t>(stream));
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

// ---------------------------------------------------------------------------
// Allocation-free variant of scn_hist_scores (see scn_hist_scores_noalloc in
// scn.h).  Its scratch lives in a fixed device array of this library instead
// of memory allocated per sequence.
// ---------------------------------------------------------------------------
namespace scn {
namespace {

constexpr int64_t kNoAllocMaxElems = 16384;
// per element: 48 partial-histogram words + 1 done counter + 1 pair counter;
// then the status word and the work-queue counters
constexpr int64_t kNoAllocWords = kNoAllocMaxElems * 50 + 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

}  // namespace
}  // namespace scn

extern "C" scn_status scn_hist_scores_noalloc(const uint8_t* d_nv12, int32_t width, int32_t height,
                                              int64_t frame_stride, const int32_t* d_slots, int64_t n,
                                              uint32_t* d_hist, uint32_t* d_score, uint8_t* d_flag, void* stream) {
    using namespace scn;
    if (n < 0) return SCN_EINVAL;
    if (n > kNoAllocMaxElems) return SCN_ERANGE;
    if (n == 0) return SCN_OK;
    if (width < 16 || height < 2 || (width % 16) || (height % 2)) return SCN_EINVAL;
    const int64_t fb = static_cast<int64_t>(width) * height * 3 / 2;
    if (frame_stride < fb || (frame_stride % 16)) return SCN_EINVAL;
    if (!d_nv12 || !aligned16(d_nv12) || !d_slots || !d_hist || !d_score || !d_flag) return SCN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_slots) & 3u) || (reinterpret_cast<uintptr_t>(d_hist) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_score) & 3u))
        return SCN_EINVAL;
    int dev = 0;
    SCN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SCN_EUNSUPPORTED;
    if (!g_noalloc_ptr[dev]) {
        // once per device, with that device current: the host-side name of the
        // array is not a device address, so ask the runtime for it
        void* p = nullptr;
        SCN_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    // the launch shape of the regular entry point, from a stack-only description
    scn_table t;
    t.W = width;
    t.H = height;
    t.num_frames = n;
    t.frame_stride = frame_stride;
    t.d_nv12 = d_nv12;
    scn_seq q;
    q.table = &t;
    q.n = n;
    const HistShape sh = resolve_hist_shape(&q);
    // scratch of this call: partial [n][48], done [n], pair [n], status, queue; zeroed first
    uint32_t* base = g_noalloc_ptr[dev];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SCN_CUDA_TRY(cudaMemsetAsync(base, 0, static_cast<size_t>(n * 50 + 8) * sizeof(uint32_t), st));
    Launch L = single_launch(&t, n, d_slots, sh);
    L.job0.hist = d_hist;
    L.job0.score = d_score;
    L.job0.flag = d_flag;
    L.job0.partial = base;
    L.job0.done = base + n * 48;
    L.job0.pair = base + n * 49;
    L.status = reinterpret_cast<int*>(base + n * 50);
    L.queue = base + n * 50 + 2;  // 8-byte aligned: (n * 50 + 2) * 4 is a multiple of 8
    return launch_hist(L, st);
}
