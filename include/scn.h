/*
 * scn.h - C ABI of the B300 sampled-frame video-analysis library (libscn.so).
 *
 * The calls follow the paper's model (Scanner, Poms et al., ACM TOG 37(4) 2018):
 * a video is a table with one row per frame (Sec. 3, "Videos as logical
 * tables"); a sampling op selects rows by stride, range or index list
 * (Sec. 3.2, "Sampling/spacing operations", and the access patterns of
 * Sec. 5.1.1); map ops run per element (Sec. 3.2, "Maps"); the shot score is a
 * stencil over two consecutive elements (Sec. 3.2, "Stencil operations") of a
 * per-frame colour histogram (Sec. 5.1.2, HIST; Sec. 5.2 shot detection from
 * histogram differences).
 *
 * Conventions
 *  - Every call returns scn_status.  Argument errors are detected on the host,
 *    before any launch, and nothing is written.  scn_status_str() gives text;
 *    scn_last_cuda_error() gives the CUDA error code behind SCN_ECUDA.
 *  - "d_" pointers are device memory owned by the caller (e.g. torch tensors),
 *    "h_" pointers are host memory.  Opaque handles (scn_video, scn_table,
 *    scn_seq) are owned by the library and freed by their *_destroy call.
 *  - A table BORROWS the caller's NV12 device buffer: it must outlive the table
 *    and every sequence sampled from it.
 *  - Compute calls are asynchronous on the given stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream).  Device-side faults that the
 *    kernels detect themselves (a bounded wait that ran out) are recorded in the
 *    sequence's status word, read by scn_seq_sync_status().
 *  - A sequence carries device scratch (completion counters and cross-CTA
 *    partial histograms, left zeroed by every call); two calls on the same
 *    sequence must not overlap on the GPU (use one stream per sequence).
 *  - Object creation (scn_video_create, scn_sample, scn_plan_create) returns
 *    once the object's device memory is filled, but does not wait for kernels
 *    already running on other streams: that memory comes from a library pool
 *    (grown ahead in large steps, kept until the process exits) and is filled
 *    by copies on a library stream.  *_destroy first waits for the device, as
 *    cudaFree does, so a sequence may be destroyed right after its last call.
 *  - Layouts: NV12 frame = W*H luma bytes then H/2 rows of W interleaved U,V
 *    bytes; histogram = uint32 [n][3][16] (R, G, B; bin = value >> 4);
 *    score = uint32 [n]; flag = uint8 [n]; resize output = [n][3][oh][ow].
 */
#ifndef SCN_H
#define SCN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SCN_OK = 0,
    SCN_EINVAL = 1,        /* bad argument: null pointer, bad size, misalignment */
    SCN_ERANGE = 2,        /* an index or size outside the table / a buffer */
    SCN_ENOMEM = 3,        /* host or device allocation failed */
    SCN_ECUDA = 4,         /* a CUDA runtime call failed (see scn_last_cuda_error) */
    SCN_ETIMEOUT = 5,      /* a bounded device wait ran out (see scn_seq_sync_status) */
    SCN_EUNSUPPORTED = 6   /* no usable sm_103 device, or an unsupported request */
} scn_status;

/* Text for a status code; never NULL. */
const char* scn_status_str(scn_status s);
/* The cudaError_t value of the last failing CUDA call made by this thread. */
int scn_last_cuda_error(void);
/* Library version string. */
const char* scn_version(void);
/* Number of SMs of the current device, or -1 without a device. */
int scn_device_sm_count(void);

/* ------------------------------------------------------------------------ */
/* Synthetic video generator (stands in for decoded frames; the paper's     */
/* compressed-video decode, Sec. 4.3, is out of scope).  SplitMix64 counter */
/* stream; shots with a base colour, a linear ramp drifting 1 px/frame and  */
/* Irwin-Hall noise of sigma 8.  The CPU oracle implements the same         */
/* definition separately; the bytes are checked equal.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t master_seed;
    uint64_t video_id;
    int32_t width, height;   /* even; width % 16 == 0 */
    int64_t num_frames;      /* >= 1 */
    int32_t num_shots;       /* shot_mode 0: shots S, 1 <= S <= num_frames */
    int32_t shot_mode;       /* 0: S-1 uniform boundaries; 1: geometric lengths (p = 1/64, 2..300) */
} scn_gen_params;

typedef struct {
    int64_t start;           /* first frame of the shot */
    int32_t base[3];         /* Y, U, V base levels */
    int32_t gx[3], gy[3];    /* ramp amplitudes per plane, in [-32, 32] */
} scn_shot;

typedef struct scn_video scn_video;

/* Host only: the shot table the generator uses for params (no device call).
 * Writes min(cap, n) shots to h_out and the full count to *n.  Errors:
 * SCN_EINVAL for bad params. */
scn_status scn_gen_shots(const scn_gen_params* params, scn_shot* h_out, int64_t cap, int64_t* n);

/* Build the shot table on the host and upload it (done on return; no wait for
 * running kernels).  Errors: SCN_EINVAL (bad params), SCN_ENOMEM, SCN_ECUDA. */
scn_status scn_video_create(const scn_gen_params* params, scn_video** out);
scn_status scn_video_destroy(scn_video* v);
/* Number of shots; copy of the first min(cap, n) shots into h_out. */
scn_status scn_video_shots(const scn_video* v, scn_shot* h_out, int64_t cap, int64_t* n);
/* Default keyframe list: every 104th frame (the paper's average keyframe
 * distance, Sec. 5.1.1) plus every shot start, ascending.  Writes
 * min(cap, n) entries into h_out and the full count into *n. */
scn_status scn_video_keyframes(const scn_video* v, int64_t* h_out, int64_t cap, int64_t* n);
/* Generate frames first_frame .. first_frame+count-1 into d_out, frame k at
 * d_out + k*frame_stride (frame_stride >= W*H*3/2, % 16 == 0; d_out 16-byte
 * aligned, else SCN_EINVAL; frames outside the video, or a frame of 2^31 or
 * more 16-byte vectors: SCN_ERANGE).  Asynchronous on stream. */
scn_status scn_generate(const scn_video* v, uint8_t* d_out, int64_t first_frame, int64_t count,
                        int64_t frame_stride, void* stream);
/* Sparse materialisation: generate frame d_frames[k] (device int64 array of n
 * frame numbers) into d_out + k*frame_stride. */
scn_status scn_generate_frames(const scn_video* v, const int64_t* d_frames, int64_t n, uint8_t* d_out,
                               int64_t frame_stride, void* stream);

/* ------------------------------------------------------------------------ */
/* Tables and sampling                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t width, height;        /* even, width % 16 == 0 */
    int64_t num_frames;           /* logical rows (frames) of the video */
    int64_t frame_stride;         /* bytes between stored frames, >= W*H*3/2, % 16 == 0 */
    const uint8_t* d_nv12;        /* device, borrowed, 16-byte aligned */
    const int64_t* h_rows;        /* optional (NULL = dense): ascending logical frame number of
                                     each stored frame; only these rows are materialised */
    int64_t num_rows;             /* entries of h_rows (ignored when h_rows is NULL) */
    const int64_t* h_keyframes;   /* optional keyframe list (copied, sorted, deduplicated) */
    int64_t num_keyframes;
} scn_table_desc;

typedef struct scn_table scn_table;
typedef struct scn_seq scn_seq;

/* Record a table over the caller's NV12 buffer (host only, no device call).
 * Errors: SCN_EINVAL for odd sizes, width % 16, stride, alignment, unsorted
 * h_rows or keyframes outside [0, num_frames). */
scn_status scn_table_create(const scn_table_desc* desc, scn_table** out);
scn_status scn_table_destroy(scn_table* t);

typedef enum {
    SCN_STRIDE = 0,     /* start, start+step, ... < stop */
    SCN_RANGE = 1,      /* [start, stop) */
    SCN_GATHER = 2,     /* h_indices[0..n), in the given order, duplicates kept */
    SCN_KEYFRAME = 3    /* the table's keyframe list */
} scn_sample_kind;

typedef struct {
    int32_t kind;                 /* scn_sample_kind */
    int64_t start, stop, step;    /* STRIDE / RANGE */
    const int64_t* h_indices;     /* GATHER (host) */
    int64_t n;                    /* GATHER length */
} scn_sample_spec;

/* Host-only: the logical frame numbers the spec selects (Sec. 3.2 sampling).
 * Writes min(cap, n) entries and sets *n.  Errors: SCN_EINVAL (bad kind, step
 * < 1), SCN_ERANGE (a row outside [0, num_frames) or not materialised). */
scn_status scn_sample_indices(const scn_table* t, const scn_sample_spec* spec, int64_t* h_out,
                              int64_t cap, int64_t* n);
/* Create a sequence: the selected rows' storage slots uploaded to the device
 * plus the sequence's zeroed scratch (about 204 bytes per element, from the
 * library's object pool; freed by scn_seq_destroy).  Returns once both are on
 * the device; does not wait for running kernels. */
scn_status scn_sample(const scn_table* t, const scn_sample_spec* spec, scn_seq** out);
scn_status scn_seq_length(const scn_seq* s, int64_t* n);
scn_status scn_seq_destroy(scn_seq* s);
/* Synchronise stream, read and clear the sequence's device status word.
 * Returns SCN_OK or SCN_ETIMEOUT.  On SCN_ETIMEOUT it also zeroes the
 * sequence's kernel scratch (cross-CTA partial histograms, frame and pair
 * counters, work queue) and its gated-path workspace, which a launch that gave
 * up may have left part-way, so the next call on the sequence starts clean;
 * the outputs of the launch that timed out are undefined. */
scn_status scn_seq_sync_status(scn_seq* s, void* stream);
/* Test hook for the bounded device waits (the paper has no counterpart; it
 * exercises the status-word path of the conventions above without faulting or
 * hanging the GPU).  Later scn_hist / scn_hist_scores launches of this sequence
 * wait at most wait_limit_ns at each bounded wait (0 restores the default 2 s;
 * otherwise it must lie in [1e5, 1e10] ns, else SCN_EINVAL), and with
 * withhold_after = k >= 0 each counting region of each CTA hands its warps k
 * chunks of work and then withholds the rest, so the waits on it run out: the
 * launch ends by itself with SCN_ETIMEOUT in the status word and undefined
 * outputs.
 * withhold_after < 0 restores normal operation.  Host-only setter. */
scn_status scn_seq_set_wait_test(scn_seq* s, uint64_t wait_limit_ns, int32_t withhold_after);

/* ------------------------------------------------------------------------ */
/* Launch shape of the fused kernel (chosen automatically when a field is 0). */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t chunk_rows;    /* luma rows per staged chunk (even), 0 = largest that fits */
    int32_t grid;          /* CTAs (one per SM at most is resident), 0 = one per SM */
    int32_t item_kpx;      /* target kilo-pixels per work item (a frame or part of one), 0 = automatic */
} scn_tune;

scn_status scn_seq_set_tune(scn_seq* s, const scn_tune* tune);
scn_status scn_seq_get_tune(const scn_seq* s, scn_tune* tune);

/* ------------------------------------------------------------------------ */
/* Per-frame ops                                                             */
/* ------------------------------------------------------------------------ */
/* d_hist[k] = 3x16-bin histogram of the BT.601 fixed-point RGB of sampled
 * frame k (R = clamp((298(Y-16) + 409(V-128) + 128) >> 8), G with -100, -208,
 * B with 516; chroma nearest; bin = v >> 4).  n = 0 writes nothing. */
scn_status scn_hist(scn_seq* s, uint32_t* d_hist, void* stream);
/* Shot scores from histograms: d_score[0] = 0, d_score[k] = L1 distance of
 * hist[k] and hist[k-1]; d_flag[k] = (2*score > pixel_count). */
scn_status scn_shot_scores(const uint32_t* d_hist, int64_t n, int64_t pixel_count, uint32_t* d_score,
                           uint8_t* d_flag, void* stream);
/* Fused: histograms and shot scores of the sequence in one launch. */
scn_status scn_hist_scores(scn_seq* s, uint32_t* d_hist, uint32_t* d_score, uint8_t* d_flag,
                           void* stream);

/* Allocation-free form of scn_hist_scores, for callers that cannot allocate
 * device memory: code running where cudaMalloc is off limits (an allocator
 * hook, a host that owns every device buffer and hands out fixed regions,
 * real-time paths that must not touch the allocator).  The paper has no
 * counterpart; this is a property of the library only.
 *   d_nv12: device frames, frame s at d_nv12 + s*frame_stride (16-byte aligned,
 *   frame_stride >= W*H*3/2 and % 16 == 0); d_slots: device int32 [n], the
 *   frame of each sampled element (every slot must name a stored frame; they are
 *   not checked); outputs as scn_hist_scores.
 * It uses a fixed scratch array inside the library, sized for at most 16384
 * elements (about 3.3 MB, held on every GPU that loads the library until the
 * process exits): n > 16384 returns SCN_ERANGE, n = 0 writes nothing.  It
 * calls no allocating routine.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  Each call clears the part of the
 * array it uses (an async memset on stream) and then launches the kernel.  All
 * calls share the one array: calls that overlap on the GPU (different streams
 * without ordering) race and give wrong results.  A device-side wait timeout
 * is recorded in the array but not reported. */
scn_status scn_hist_scores_noalloc(const uint8_t* d_nv12, int32_t width, int32_t height, int64_t frame_stride,
                                   const int32_t* d_slots, int64_t n, uint32_t* d_hist, uint32_t* d_score,
                                   uint8_t* d_flag, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched plans: many sequences (of any tables, resolutions, lengths and    */
/* sampling patterns) histogrammed and scored by ONE persistent launch fed   */
/* by a device work queue of (sequence, frame, row-range) items - the        */
/* paper's work packets distributed over graph instances (Sec. 4.1).         */
/* ------------------------------------------------------------------------ */
typedef struct scn_plan scn_plan;

/* Build a plan over nseq distinct sequences with their outputs (device,
 * caller-owned; entry i as in scn_hist_scores for seqs[i]).  tune may be NULL
 * (automatic shapes).  Uploads the job and item lists (done on return; no wait
 * for running kernels).  The
 * sequences' scratch is used by the plan's launches: do not run a sequence
 * and a plan containing it concurrently.  Errors: SCN_EINVAL (NULL entries,
 * repeated sequence, misaligned outputs), SCN_ECUDA. */
scn_status scn_plan_create(scn_seq* const* seqs, int32_t nseq, uint32_t* const* d_hist, uint32_t* const* d_score,
                           uint8_t* const* d_flag, const scn_tune* tune, scn_plan** out);
scn_status scn_plan_destroy(scn_plan* p);
/* Change the launch shape (rebuilds the item list, drops a captured graph). */
scn_status scn_plan_set_tune(scn_plan* p, const scn_tune* tune);
scn_status scn_plan_get_tune(const scn_plan* p, scn_tune* tune);
/* Work items, sampled frames, NV12 bytes read per run, and CTAs of a run. */
scn_status scn_plan_info(const scn_plan* p, int64_t* n_items, int64_t* n_frames, int64_t* nv12_bytes, int32_t* grid);
/* One asynchronous run on stream. */
scn_status scn_plan_run(scn_plan* p, void* stream);
/* Capture one run into a CUDA graph owned by the plan (stream must not be the
 * legacy default stream); scn_plan_replay launches it. */
scn_status scn_plan_capture_graph(scn_plan* p, void* stream);
scn_status scn_plan_replay(scn_plan* p, void* stream);
/* Synchronise stream, read and clear the plan's device status word; on
 * SCN_ETIMEOUT also zero the plan's work queue and the kernel scratch of each
 * of its sequences (see scn_seq_sync_status). */
scn_status scn_plan_sync_status(scn_plan* p, void* stream);
/* Autotuner: time candidate shapes (item size x chunk rows) with `reps`
 * runs each on stream (synchronous), keep the fastest; returns it and its
 * mean time per run (either pointer may be NULL).  Outputs are overwritten by
 * identical results. */
scn_status scn_plan_autotune(scn_plan* p, int32_t reps, void* stream, scn_tune* best, float* best_ms);

/* ------------------------------------------------------------------------ */
/* Learned boundary proposal: a tiny BF16 CNN (FP32 accumulation, tcgen05    */
/* tensor cores for the convolutions) over pairs of 36x64 luma thumbnails.    */
/* The paper runs DNNs on sampled frames (Sec. 3.1, Sec. 5.1.2) but fixes no   */
/* proposal network; this library's is:                                     */
/*   x = [(Yprev-128)/64, (Ycur-128)/64] (2x36x64) -> conv3x3/s2/p1 2->16 ->  */
/*   16->32 -> 32->32 (each + bias + ReLU) -> mean over 5x8 -> FC 32->64 +    */
/*   ReLU -> FC 64->1 = logit.  16369 parameters, flat fp32 in that order    */
/*   (conv weights [co][ci][3][3]).                                          */
/* ------------------------------------------------------------------------ */
typedef struct scn_cnn scn_cnn;

/* Number of parameters (16369). */
int64_t scn_cnn_num_params(void);
/* Allocate a network with room for max_batch pairs per launch (activations,
 * gradients, Adam state).  Parameters start at zero: set them first. */
scn_status scn_cnn_create(int64_t max_batch, scn_cnn** out);
scn_status scn_cnn_destroy(scn_cnn* c);
/* Copy n = scn_cnn_num_params() fp32 parameters from the host; resets the
 * optimiser state.  Synchronous. */
scn_status scn_cnn_set_params(scn_cnn* c, const float* h_params, int64_t n);
scn_status scn_cnn_get_params(const scn_cnn* c, float* h_params, int64_t n);
/* Logits of n thumbnail pairs (any n; inference, Sec. 5.1.2 DNN over sampled
 * frames).  d_thumbs: uint8 [*][36][64] (device, 16-byte aligned, else
 * SCN_EINVAL).  Pair b is (d_prev[b], d_cur[b]) (device int32 thumbnail
 * indices, which the caller keeps inside the thumbnail array) or, when both are
 * NULL, (b, b+1).  One launch of a fused kernel that keeps every activation on
 * chip; it stores no activations (scn_cnn_activation shows the last training
 * batch). */
scn_status scn_cnn_forward(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                           int64_t n, float* d_logits, void* stream);
/* Gradients of the batch-mean BCE-with-logits loss (positive weight
 * pos_weight > 0) over `batch` pairs (1..max_batch) with labels d_labels
 * (device float 0/1): d_grads (device, num_params floats, parameter order) and
 * d_loss (device float); either may be NULL.  Gradients are taken w.r.t. the
 * BF16 weights the forward uses. */
scn_status scn_cnn_gradients(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                             const float* d_labels, int64_t batch, float pos_weight, float* d_loss, float* d_grads,
                             void* stream);
/* One training step: gradients as above, then Adam (beta 0.9 / 0.999, eps
 * 1e-8, bias-corrected) on the fp32 master weights and a refresh of the BF16
 * copies.  Asynchronous on stream. */
scn_status scn_cnn_train_step(scn_cnn* c, const uint8_t* d_thumbs, const int32_t* d_prev, const int32_t* d_cur,
                              const float* d_labels, int64_t batch, float pos_weight, float lr, float* d_loss,
                              void* stream);
/* Device pointer to the BF16 NHWC output of conv layer 1, 2 or 3 of the last
 * scn_cnn_gradients / scn_cnn_train_step batch ([pairs][positions][channels]). */
scn_status scn_cnn_activation(const scn_cnn* c, int32_t layer, const void** d_ptr);
/* Synchronise stream, read and clear the network's device status word.
 * Returns SCN_OK or SCN_ETIMEOUT (a bounded wait of a launch ran out; that
 * launch's outputs are undefined; the network keeps no scratch between
 * launches, so the next call is unaffected). */
scn_status scn_cnn_sync_status(scn_cnn* c, void* stream);
/* Test hook for the inference kernel's bounded waits (no counterpart in the
 * paper; it exercises the status-word path without faulting or hanging the
 * GPU).  Later scn_cnn_forward launches (and the learned / cascade paths that
 * run them) wait at most wait_limit_ns at each bounded wait (0 restores the
 * default 2 s; otherwise it must lie in [1e5, 1e10] ns, else SCN_EINVAL), and
 * with withhold_batch = k >= 0 every CTA's builder warps withhold the "input
 * built" signal of their k-th batch, so the waits on it run out: the launch
 * ends by itself with SCN_ETIMEOUT in the status word and undefined logits.
 * withhold_batch < 0 restores normal operation.  Host-only setter. */
scn_status scn_cnn_set_wait_test(scn_cnn* c, uint64_t wait_limit_ns, int32_t withhold_batch);

/* ------------------------------------------------------------------------ */
/* Spacing and slicing (Sec. 3.2) and the per-shot montage (Sec. 5.2)       */
/* ------------------------------------------------------------------------ */
typedef enum {
    SCN_FILL_VALUE = 0,    /* frames no element samples get the fill element */
    SCN_FILL_REPEAT = 1    /* ... the output of the nearest earlier sampled frame (fill before the first) */
} scn_fill_mode;

/* Spacing, the inverse of the sampling op that made s (Sec. 3.2, "Sampling/
 * spacing operations": fill elements align sequences sampled at different
 * rates).  d_in: n = length(s) elements of elem_bytes bytes (1..1024), device,
 * element k being the result for sampled frame k of s.  d_out: num_frames
 * elements of the table (device): element t = the input element whose sampled
 * frame is t (the last such element when s samples t more than once); frames
 * that no element samples get h_fill (elem_bytes bytes, host; NULL = zero
 * bytes) or, with SCN_FILL_REPEAT, the element of the nearest earlier sampled
 * frame.  The first call on a sequence builds its sorted frame list on the
 * device (synchronous); later calls are asynchronous on stream.  Errors:
 * SCN_EINVAL (bad size or mode, NULL buffers), SCN_ERANGE (more than 2^31-1
 * frames), SCN_ECUDA. */
scn_status scn_space(scn_seq* s, const void* d_in, int32_t elem_bytes, int32_t fill_mode, const void* h_fill,
                     void* d_out, void* stream);

/* Slicing at boundaries (Sec. 3.2, "Slicing/unslicing operations": e.g. at
 * shot boundaries, so that stencils and state do not cross shots): element k
 * of an n-element sequence starts a slice when k == 0 or d_flag[k] != 0 (for
 * instance the shot flags of scn_hist_scores).  d_start (device int32,
 * capacity n) receives the first element of every slice in ascending order,
 * d_count (device int64) the number of slices.  n = 0 writes count 0.
 * Errors: SCN_EINVAL, SCN_ERANGE (n > 2^31-1). */
scn_status scn_slice(const uint8_t* d_flag, int64_t n, int32_t* d_start, int64_t* d_count, void* stream);
/* One representative element per slice (the film summaries of Sec. 5.2 show
 * one frame per shot): d_mid[i] = (start[i] + end[i] - 1) / 2, end[i] =
 * start[i+1] or n, for i < *d_count (read on the device). */
scn_status scn_slice_middles(const int32_t* d_start, const int64_t* d_count, int64_t n, int32_t* d_mid, void* stream);
/* Shot scores whose two-element stencil stops at slice boundaries: score[k]
 * = 0 where a slice starts (k == 0 or d_boundary[k] != 0, device uint8 [n]),
 * else as scn_shot_scores. */
scn_status scn_shot_scores_sliced(const uint32_t* d_hist, int64_t n, int64_t pixel_count, const uint8_t* d_boundary,
                                  uint32_t* d_score, uint8_t* d_flag, void* stream);
/* Stencil S[a, b] over a histogram sequence (Sec. 3.2, "Stencil operations":
 * an op may read a window of elements around each one), the windowed shot
 * score: with P = -a frames before element k and F = b + 1 frames from it
 * (-64 <= a < 0 <= b < 64),
 *   score[k] = sum over the 48 bins |F * sum_{j=a}^{-1} h[k+j] - P * sum_{j=0}^{b} h[k+j]|
 *   flag[k]  = 2 * score[k] > P * F * pixel_count
 * (the L1 distance of the two windows' mean histograms, scaled by P*F to stay
 * integer; a = -1, b = 0 is scn_shot_scores).  k whose window leaves [0, n), or
 * holds a slice start after its first frame (d_boundary != 0 at k+a+1 .. k+b;
 * d_boundary may be NULL), gets 0.  Only a slice of the sequence need be
 * resident: d_hist (device uint32 [hist_count][48]) and d_boundary hold
 * elements [hist_first, hist_first + hist_count); the outputs are elements
 * [k0, k1), written to d_score[k - k0] (device uint64) and d_flag[k - k0].  The
 * outputs' dependency range (Sec. 4.2), [max(0, k0 + a), min(n, k1 + b)), must
 * lie inside the resident slice, else SCN_ERANGE: a sequence can be split into
 * shards that each carry their -a / b element halo.  Errors: SCN_EINVAL. */
scn_status scn_window_scores(const uint32_t* d_hist, int64_t hist_first, int64_t hist_count, int64_t n, int32_t a,
                             int32_t b, int64_t pixel_count, const uint8_t* d_boundary, int64_t k0, int64_t k1,
                             uint64_t* d_score, uint8_t* d_flag, void* stream);
/* Bounded-state shot score (Sec. 3.2, "Bounded state operations": an op may
 * carry state from element to element, and before it produces element i it
 * has processed at least the `warmup` elements before i).  The state is a
 * reference histogram m.  The first element a run processes, and an element
 * where a slice starts (d_boundary != 0; d_boundary may be NULL), set m to its
 * histogram h and output score 0, flag 0.  Every other element outputs
 *   score = sum over the 48 bins |h - m|,  flag = 2 * score > pixel_count,
 * then sets m = h if flag (a cut restarts the reference) else
 * m += floor((h - m) / 2^shift) (an exponential average of the shot so far);
 * shift = 0 gives the plain two-frame score.
 * Runs: run r (0 <= r < runs) has outputs [k0, k1) = [run_first + r*run_stride,
 * + run_len) clipped to [0, n), processed on its own from max(0, k0 - warmup);
 * element k of run r goes to d_score[r*run_len + k - k0] (device uint32) and
 * d_flag[...]; slots of elements past n are not written.  One run of n
 * outputs is the serial op; run_len == run_stride splits it into shards;
 * run_len 1 produces sparse outputs, each after `warmup` elements.  Results
 * depend on the runs chosen (as the paper allows for bounded state), and equal
 * the serial op's where a run's warmup reaches back to a slice start or to 0.
 * d_hist (device uint32 [hist_count][48], as scn_hist writes it: each channel
 * sums to pixel_count) and d_boundary hold elements [hist_first, hist_first +
 * hist_count), which must cover [max(0, run_first - warmup), end of the last
 * run) (Sec. 4.2: warmup W is the footprint i - W .. i), else SCN_ERANGE.
 * Errors: SCN_EINVAL (shift outside 0..30, warmup < 0, run_len < 1,
 * run_stride < run_len, ...), SCN_ERANGE (pixel_count > 715827882). */
scn_status scn_bounded_state_scores(const uint32_t* d_hist, int64_t hist_first, int64_t hist_count, int64_t n,
                                   int64_t pixel_count, int32_t shift, int64_t warmup, int64_t run_first,
                                   int64_t run_len, int64_t run_stride, int64_t runs, const uint8_t* d_boundary,
                                   uint32_t* d_score, uint8_t* d_flag, void* stream);
/* Montage of sequence elements (Sec. 5.2, film summaries: one frame from each
 * shot): tile i (row-major, `cols` tiles per row) shows element d_elem[i]
 * (device int32, m entries) of s, nearest-neighbour downsampled to tile_w x
 * tile_h (1..4096): tile pixel (x, y) = BT.601 fixed-point RGB (as scn_hist)
 * of source pixel (floor((2x+1) W / (2 tile_w)), floor((2y+1) H / (2 tile_h))).
 * d_out: uint8 [rows*tile_h][cols*tile_w][3], rows = ceil(m / cols), device;
 * tiles past m, and tiles whose element is outside s, are black.  m = 0 writes
 * nothing.  Errors: SCN_EINVAL, SCN_ERANGE (more than 2^34 output pixels). */
scn_status scn_montage(const scn_seq* s, const int32_t* d_elem, int64_t m, int32_t cols, int32_t tile_w,
                       int32_t tile_h, uint8_t* d_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Gated exact path: a gate proposes boundary candidates, only the frames of */
/* proposed pairs go through the exact kernel, which keeps the final say.  */
/* ------------------------------------------------------------------------ */
/* d_gate[k] (device float, k >= 1) scores pair (k-1, k) of the sequence; pair
 * k is proposed when d_gate[k] > tau (d_gate[0] is ignored).  Writes
 * d_proposed[k] (0/1); d_score / d_flag get the exact score and flag of every
 * proposed pair and 0 elsewhere.  The number of proposals stays on the device
 * (every launch reads it there), so with h_nproposed NULL the call is fully
 * asynchronous on stream; when h_nproposed is not NULL the call waits for the
 * stream at its end and writes the number there.  The sequence's gated
 * workspace is allocated on the first call (synchronous). */
scn_status scn_gated_hist_scores(scn_seq* s, const float* d_gate, float tau, uint8_t* d_proposed, uint32_t* d_score,
                                 uint8_t* d_flag, int64_t* h_nproposed, void* stream);
/* The learned proposal path: thumbnails of the sequence into d_thumbs
 * (caller-owned [n][36][64]), the network's logit of every consecutive pair
 * into d_logits[1..n-1] (pair k-1, k), then scn_gated_hist_scores with tau. */
scn_status scn_proposal_hist_scores(scn_seq* s, scn_cnn* net, float tau, uint8_t* d_thumbs, float* d_logits,
                                    uint8_t* d_proposed, uint32_t* d_score, uint8_t* d_flag, int64_t* h_nproposed,
                                    void* stream);
/* The non-learned gate: d_diff[k] = mean |thumb[k] - thumb[k-1]| over the
 * 2304 samples (d_diff[0] = 0); d_thumbs 4-byte aligned. */
scn_status scn_thumb_diff(const uint8_t* d_thumbs, int64_t n, float* d_diff, void* stream);
/* The luma + chroma gate over coarse YUV thumbnails (scn_thumbs_yuv): d_diff[k]
 * = mean |dY| + mean |dU| + mean |dV| between elements k-1 and k, 192 samples
 * per plane (d_diff[0] = 0).  d_yuv [n][3][6][32], 16-byte aligned, else
 * SCN_EINVAL.  A boundary that changes chroma but little luma still moves it. */
scn_status scn_thumb_diff_yuv(const uint8_t* d_yuv, int64_t n, float* d_diff, void* stream);
/* The cascade: the luma + chroma gate as a cheap prefilter, the network on what
 * it passes.  Coarse YUV thumbnails of every element into d_yuv
 * ([n][3][6][32], 16-byte aligned) and the gate (scn_thumb_diff_yuv) into
 * d_diff ([n]); the network's luma thumbnails into d_thumbs ([n][36][64],
 * 16-byte aligned) for the two elements of each pair whose gate passes
 * tau_diff only (other entries are not written); every pair with d_diff[k] > tau_diff
 * gets the network's logit in d_gate[k], every other pair -infinity; then
 * scn_gated_hist_scores with tau_net, so a pair is proposed only when both
 * thresholds pass and the exact kernel keeps the final say.  The network runs
 * on the listed pairs only (their count stays on the device: no host round
 * trip).  Workspace as scn_gated_hist_scores.  d_diff, d_gate, d_score 4-byte
 * aligned (SCN_EINVAL); more than 2^31 - 1 elements: SCN_ERANGE. */
scn_status scn_cascade_hist_scores(scn_seq* s, scn_cnn* net, float tau_diff, float tau_net, uint8_t* d_thumbs,
                                   uint8_t* d_uv, float* d_diff, float* d_gate, uint8_t* d_proposed,
                                   uint32_t* d_score, uint8_t* d_flag, int64_t* h_nproposed, void* stream);

typedef enum { SCN_F32 = 0, SCN_BF16 = 1 } scn_dtype;
/* Bilinear resize (half-pixel centres, no antialias, stretch) of the RGB
 * frame to oh x ow, then (v/255 - mean[c]) / std[c]; output [n][3][oh][ow]
 * in dtype.  mean/std are host arrays of 3. */
scn_status scn_resize_norm(scn_seq* s, int32_t oh, int32_t ow, const float* h_mean, const float* h_std,
                           int32_t dtype, void* d_out, void* stream);
/* The same resize and normalisation written once as FP32 (d_out_f32) and once
 * as BF16 (d_out_bf16, the RNE of each FP32 value), from one pass over the
 * source rows: the two layouts of the two scn_resize_norm calls, for half the
 * reads.  Both outputs [n][3][oh][ow], device, 4- and 2-byte aligned. */
scn_status scn_resize_norm_both(scn_seq* s, int32_t out_h, int32_t out_w, const float* h_mean, const float* h_std,
                                float* d_out_f32, void* d_out_bf16, void* stream);
/* Luma thumbnails: d_thumb[k][r][c] = Y[s*r][s*c], s = W/64 = H/36
 * (requires W == 64*s and H == 36*s); output uint8 [n][36][64]. */
scn_status scn_thumbs(scn_seq* s, uint8_t* d_thumb, void* stream);
/* Coarse YUV thumbnails and, in the same launch when d_thumb is not NULL, the
 * luma thumbnails of scn_thumbs: d_yuv[k][0][r][c] = Y[6*s*r][2*s*c] and
 * d_yuv[k][1][r][c], d_yuv[k][2][r][c] = U, V of chroma sample (s*c, 3*s*r),
 * the one under that luma pixel, r < 6, c < 32; output uint8 [n][3][6][32]
 * (NULL: luma thumbnails only; both NULL: SCN_EINVAL). */
scn_status scn_thumbs_yuv(scn_seq* s, uint8_t* d_thumb, uint8_t* d_yuv, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SCN_H */
