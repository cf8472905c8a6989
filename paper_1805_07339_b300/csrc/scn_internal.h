// Internal declarations shared by the libscn translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// Device status word bits (per sequence).
constexpr int kStatusTimeout = 1;

// Histogram kernel geometry (fixed at compile time).
constexpr int kConsumerWarps = 16;                        // warps that convert + count
constexpr int kHistThreads = (kConsumerWarps + 1) * 32;  // + one producer warp (bulk copies)
constexpr int kStages = 2;                                // staged chunks in flight (2 x ~30 KB measured best)
constexpr int kGroupWarps = 4;                            // warps sharing one table region
constexpr int kRegions = kConsumerWarps / kGroupWarps;
constexpr int kTabRowsPerRegion = 136;                    // 45 (R) + 39 (G) + 52 (B) extended bins
constexpr int kTabBytes = kRegions * kTabRowsPerRegion * 256;
constexpr int kSmemLimit = 232448;                        // 227 KB opt-in per CTA
constexpr int kSmemMisc = 1024;                           // accumulators + barriers + flags
constexpr int kStageBudget = (kSmemLimit - kTabBytes - kSmemMisc) / kStages;
// Pixels a CTA may count between two table flushes: keeps every 16-bit lane
// counter below 2^16 (each of the 512 consumer threads sees at most 1/512 of them).
constexpr int64_t kSegmentPixels = int64_t(1) << 24;

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
    scn_tune tune{0, 0, 0};          // 0 fields: chosen per call
};

namespace scn {
// Launch shape resolved for a sequence (see scn_hist.cu).
struct HistShape {
    int chunk_rows;      // luma rows per staged chunk (even)
    int grid;            // CTAs
    int stage_bytes;     // bytes per stage buffer
    int seg_rows;        // luma rows counted between two table flushes (even)
    int64_t rp_per_cta;  // row pairs (2 luma rows + 1 chroma row) per CTA
    size_t smem;
};
HistShape resolve_hist_shape(const scn_seq* s);
int device_sm_count();
}  // namespace scn
