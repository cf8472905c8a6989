// Internal declarations shared by the libscn translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "../../include/scn.h"

namespace scn {

// Records a failing CUDA call for scn_last_cuda_error().
void set_cuda_error(cudaError_t e);

#define SCN_CUDA_TRY(call)                        \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) {                  \
            ::scn::set_cuda_error(e_);            \
            return SCN_ECUDA;                     \
        }                                         \
    } while (0)

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Launch with programmatic stream serialization: the grid may be scheduled
// while the previous kernel in the stream is still finishing, so the launch
// latency overlaps it.  Only kernels that call ptx::pdl_wait() before their
// first global memory access are launched this way.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Runs set() once per device for the current device: `done` holds one bit per
// device (at most 64).  Safe from several host threads on different devices;
// two threads on one device may both run set(), which only repeats an
// idempotent attribute call.  Later calls cost one atomic load.
template <class F>
inline scn_status once_per_device(std::atomic<uint64_t>& done, F&& set) {
    int dev = 0;
    SCN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SCN_EUNSUPPORTED;
    const uint64_t bit = uint64_t(1) << dev;
    if (done.load(std::memory_order_acquire) & bit) return SCN_OK;
    const scn_status s = set();
    if (s == SCN_OK) done.fetch_or(bit, std::memory_order_acq_rel);
    return s;
}

// Device memory of library objects (videos, sequences, plans), in scn_mem.cu:
// from a per-device pool grown ahead in large steps and filled on a library
// stream that waits for no other stream, by copies only (a kernel would queue
// behind running grids), so creating an object does not wait for kernels
// already running.  obj_finish() waits for the fills issued so
// far; obj_free() first waits for the device, as cudaFree does.
cudaError_t obj_stream(cudaStream_t* s);
cudaError_t obj_alloc(void** p, size_t bytes);
cudaError_t obj_upload(void* dst, const void* src, size_t bytes);
cudaError_t obj_zero(void* dst, size_t bytes);
cudaError_t obj_finish();
void obj_free(void* p);

// Device status word bits (per sequence).
constexpr int kStatusTimeout = 1;

// Histogram kernel geometry (fixed at compile time).
constexpr int kConsumerWarps = 20;                        // warps that load, convert + count
constexpr int kHistThreads = (kConsumerWarps + 2) * 32;  // + a producer warp (work descriptors) + a publisher warp
constexpr int kHistThreadsRg = (kConsumerWarps + 1) * 32;  // region streams: + a publisher warp
constexpr int kStages = 2;                                // chunk descriptors in flight
constexpr int kGroupWarps = 4;                            // warps sharing one table region
constexpr int kRegions = kConsumerWarps / kGroupWarps;
constexpr int kTabRowsPerRegion = 136;                    // 45 (R) + 39 (G) + 52 (B) extended bins
constexpr int kTabBytes = kRegions * kTabRowsPerRegion * 256;
constexpr int kReductionsPerPixel = 3;                    // one shared-memory count per channel
constexpr int kSmemLimit = 232448;                        // 227 KB opt-in per CTA
constexpr int kSmemMisc = 4096;                           // accumulators, chunk descriptors, barriers, flags
static_assert(kTabBytes + kSmemMisc <= kSmemLimit, "tables fit in shared memory");
constexpr int kConsumerThreads = kConsumerWarps * 32;
// Pixels of one work item at most: the table is flushed after every item, and
// this keeps every 16-bit lane counter below 2^16 (each counter belongs to one
// consumer thread, which counts at most 1/kConsumerThreads of an item's
// pixels plus one unit of 32).
constexpr int64_t kItemPixelsMax = int64_t(1) << 24;
static_assert(kItemPixelsMax / kConsumerThreads + 2 * 32 < 65536, "16-bit lane counters");
// Frames of at most this many pixels are counted by the region-stream kernel
// (queue launches only): each 4-warp table region takes whole items of its own,
// so an item's flush reads and zeroes one region's table instead of all five
// (a fifth of the flush traffic per frame; at 640 x 360 the flush is otherwise
// an eighth of the kernel's shared-memory traffic).  Larger frames stay with
// the CTA-wide kernel, which streams one frame per SM.  One thread of the
// counting region counts at most 1/kRegionThreads of an item plus two units.
constexpr int kRegionThreads = kGroupWarps * 32;
constexpr int64_t kRegionFramePxMax = int64_t(1) << 20;
static_assert(kRegionFramePxMax / kRegionThreads + 2 * 32 < 65536, "16-bit lane counters (region streams)");
inline bool region_frames(int W, int H) { return static_cast<int64_t>(W) * H <= kRegionFramePxMax; }
constexpr int kTailParts = 4;  // parts of each of the last `grid` frames of a whole-frame queue

}  // namespace scn

struct scn_video {
    scn_gen_params p;
    std::vector<scn_shot> shots;   // host copy
    scn_shot* d_shots = nullptr;   // device copy
};

struct scn_table {
    int32_t W, H;
    int64_t num_frames;
    int64_t frame_stride;
    const uint8_t* d_nv12;
    std::vector<int64_t> rows;       // empty: dense
    std::vector<int64_t> keyframes;  // sorted, unique
};

struct scn_seq {
    const scn_table* table;
    int64_t n;
    std::vector<int64_t> frames;     // logical frame numbers (host)
    // device memory (one allocation, carved)
    void* d_block = nullptr;
    int32_t* d_slot = nullptr;       // storage slot per element [n]
    uint32_t* d_done = nullptr;      // per-element counted row pairs [n] (kept zero)
    uint32_t* d_pair = nullptr;      // per-element arrivals of the score stencil [n]
    uint32_t* d_partial = nullptr;   // [n][48] cross-CTA histogram accumulators (kept zero)
    int* d_status = nullptr;         // device status word
    uint32_t* d_queue = nullptr;     // work-queue counters (2 words, left zero)
    void* gate_ws = nullptr;         // gated-path workspace, made on first use
    void* space_ws = nullptr;        // spacing workspace (sorted sampled frames), made on first use
    size_t scratch_off = 0;          // byte offset of the kernel scratch (done .. queue) in d_block
    size_t scratch_bytes = 0;        // its size
    scn_tune tune{0, 0, 0};          // 0 fields: chosen per call
    uint64_t test_wait_ns = 0;       // scn_seq_set_wait_test: wait limit of this sequence's launches
    int32_t test_withhold = -1;      // scn_seq_set_wait_test: chunks handed out before withholding
};

namespace scn {

// One sampled sequence as the fused kernel sees it (host-filled, device-read).
struct Job {
    const uint8_t* nv12;   // frames of the table
    int64_t stride;        // bytes between stored frames
    const int32_t* slot;   // stored frame of each element [n]
    uint32_t* hist;        // [n][48]
    uint32_t* score;       // [n], null: histograms only
    uint8_t* flag;         // [n]
    uint32_t* partial;     // [n][48] cross-CTA accumulators (left zero)
    uint32_t* done;        // [n] counted row pairs (left zero)
    uint32_t* pair;        // [n] score stencil arrivals (left zero)
    const int32_t* score_at;  // null: score[k], flag[k] for every k; else only odd k, written to
                              // score[score_at[k / 2]], flag[score_at[k / 2]] (the pairs of a gated pass)
    int64_t n;
    int32_t W, H;
    int32_t chunk_rows;    // luma rows per staged chunk (even)
    int32_t item_rp;       // row pairs per work item
    int32_t items_per_frame;
    int32_t tail_from;     // tail_parts > 0 (whole-frame queues): frames from tail_from on are
    int32_t tail_parts;    // queued as tail_parts items of tail_rp row pairs each, so that the
    int32_t tail_rp;       // launch ends on parts of frames
    int32_t wv, sp, sc;    // 16-byte columns per row; consumer threads / wv; consumer threads % wv
    uint32_t dY, dU;       // luma / chroma byte step per consumer-thread stride of units
    int32_t sc_r;          // the same for one table region's threads (region-stream kernel)
    uint32_t dY_r, dU_r;
    float inv_wv;          // 1 / wv
};

// One work item: row pairs [rp0, rp0 + nrp) of element k of job `job`.
struct Item {
    int32_t job, k, rp0, nrp;
};

// Everything one launch of the fused kernel needs.
struct Launch {
    Job job0;              // the job of a single-sequence launch
    const Job* jobs;       // device array of jobs (batched plans), null: job0 only
    const Item* items;     // device array of items (batched plans), null: implicit items of job0
    int64_t n_items;
    int64_t rp_per_cta;    // > 0: no queue; CTA b takes row pairs [b*rp_per_cta, (b+1)*rp_per_cta) of job0;
                           // < 0: the same split, computed on the device from d_count over gridDim.x CTAs
    uint32_t* queue;       // [0..1] next item (64-bit), [2] CTAs done with the queue; left zero
    int* status;           // device status word
    int grid;
    // optional device-side element count of job0 (single-sequence launches):
    // when set, job0 has count_mul * (*d_count) elements and n_items is only an
    // upper bound; the count is read by the kernel, so the host need not wait for it
    const int32_t* d_count = nullptr;
    int32_t count_mul = 0;
    uint64_t wait_limit_ns = 0;   // bounded waits give up after this long (0: 2 s)
    int32_t withhold_after = -1;  // test hook, >= 0: each producer (each table region with region
                                  // streams) stops after this many chunks
    int32_t region_items = 0;     // 1: the region-stream kernel (queue launches of frames up to
                                  // kRegionFramePxMax pixels), 0: the CTA-wide kernel
};

// Luma rows per work descriptor: the requested even count, or (0) the whole
// frame, so that a descriptor covers a whole item or segment.
int chunk_rows_for(int W, int H, int requested);
// Fill the derived consumer constants of a job (wv, sp, sc, dY, dU, inv_wv).
void fill_job_consts(Job& j);
// Row pairs per item and items per frame for a job, given a target of pixels
// per item (0: automatic for n elements over grid CTAs).
void choose_items(Job& j, int64_t item_px, int grid);
// Launch the fused kernel.
scn_status launch_hist(const Launch& L, cudaStream_t st);
// One-time per-device kernel setup (shared-memory attribute); call outside stream capture.
scn_status prepare_hist();

// Launch shape resolved for a sequence.
struct HistShape {
    int chunk_rows;      // luma rows per work descriptor (even)
    int grid;            // CTAs
    int item_rp;         // row pairs per work item
    int items_per_frame;
    int64_t rp_per_cta;  // > 0: contiguous row-pair range per CTA instead of the queue
    size_t smem;
};
HistShape resolve_hist_shape(const scn_seq* s);
// A single-sequence launch over n elements with the given storage slots
// (outputs, scratch, queue and status are filled in by the caller).
Launch single_launch(const scn_table* t, int64_t n, const int32_t* slot, const HistShape& sh);
int device_sm_count();

// The fused proposal forward over pairs (d_prev[b], d_cur[b]) whose count is
// read on the device (*d_pairs, at most max_pairs): logit of pair b into
// d_logits[b], or into d_logits[d_out_index[b]] when d_out_index is given.
scn_status cnn_forward_counted(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                               int64_t max_pairs, const int* d_pairs, float* d_logits, cudaStream_t st,
                               const int32_t* d_out_index);
// Luma (d_thumb) and/or coarse YUV (d_yuv) thumbnails of every element, as
// scn_thumbs_yuv, and *zero = 0 when zero is given (scn_resize.cu).
scn_status launch_thumbs(const scn_seq* s, uint8_t* d_thumb, uint8_t* d_yuv, int* zero, cudaStream_t st);
// Luma thumbnails of both frames of listed pairs i < *count (sequence elements
// prev[i], cur[i]) into out[element] (scn_resize.cu); max_pairs bounds *count.
scn_status launch_thumbs_listed(const scn_seq* s, const int32_t* prev, const int32_t* cur, const int* count,
                                int64_t max_pairs, uint8_t* out, cudaStream_t st);
// Release a sequence's gated-path workspace (scn_proposal.cu).
void free_gate_workspace(scn_seq* s);
// Zero the gated-path workspace's kernel scratch after a device timeout, on st.
cudaError_t reset_gate_workspace(scn_seq* s, cudaStream_t st);
// Zero a sequence's kernel scratch (cross-CTA accumulators, counters, queue,
// status) and its gated-path workspace, on st: what a timed-out launch may have
// left non-zero.
cudaError_t reset_seq_scratch(scn_seq* s, cudaStream_t st);
void free_space_workspace(scn_seq* s);
}  // namespace scn
