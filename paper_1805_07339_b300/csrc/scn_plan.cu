// Batched plans: many sampled sequences (any tables, resolutions, lengths and
// sampling patterns) histogrammed and scored in one persistent launch of the
// fused kernel, fed by a device work queue of (sequence, frame, row-range)
// items, optionally captured once into a CUDA graph and replayed, with launch
// shapes chosen by a timing autotuner.
//
// Paper anchors: work packets distributed to graph instances (Sec. 4.1);
// packet sizes are tuned by hand in the paper, which notes that automatic
// tuning is possible (Sec. 4.1) - here the autotuner does it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <set>
#include <vector>

#include "scn_internal.h"

struct scn_plan {
    std::vector<scn_seq*> seqs;
    std::vector<uint32_t*> hist, score;
    std::vector<uint8_t*> flag;
    scn_tune tune{0, 0, 0};
    std::vector<scn::Job> jobs;     // host copy of the device job array
    int64_t n_items = 0;
    int grid = 0;
    void* d_block = nullptr;        // status + queue
    scn::Job* d_jobs = nullptr;
    scn::Item* d_items = nullptr;
    int64_t items_cap = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace scn {
namespace {

constexpr int64_t kPlanItemPixelsAuto = 1920LL * 1080;  // a 1080p frame per item by default

scn_status build_items(scn_plan* p) {
    int sms = device_sm_count();
    if (sms <= 0) return SCN_EUNSUPPORTED;
    const int grid_req = p->tune.grid > 0 ? p->tune.grid : sms;
    const int64_t item_px = p->tune.item_kpx > 0 ? static_cast<int64_t>(p->tune.item_kpx) * 1000 : kPlanItemPixelsAuto;
    p->jobs.assign(p->seqs.size(), Job{});
    int64_t total_frames = 0;
    bool region = true;  // every frame small enough for the region-stream kernel
    for (scn_seq* s : p->seqs) {
        total_frames += s->n;
        region = region && region_frames(s->table->W, s->table->H);
    }
    // too few items for the CTAs: split frames further
    int64_t px_target = item_px;
    for (size_t j = 0; j < p->seqs.size(); ++j) {
        const scn_seq* s = p->seqs[j];
        Job& J = p->jobs[j];
        J.nv12 = s->table->d_nv12;
        J.stride = s->table->frame_stride;
        J.slot = s->d_slot;
        J.hist = p->hist[j];
        J.score = p->score[j];
        J.flag = p->flag[j];
        J.partial = s->d_partial;
        J.done = s->d_done;
        J.pair = s->d_pair;
        J.n = s->n;
        J.W = s->table->W;
        J.H = s->table->H;
        J.chunk_rows = chunk_rows_for(J.W, J.H, p->tune.chunk_rows);
        fill_job_consts(J);
    }
    for (int pass = 0; pass < 8; ++pass) {
        int64_t items = 0;
        for (Job& J : p->jobs) {
            choose_items(J, px_target, grid_req);
            items += J.n * J.items_per_frame;
        }
        p->n_items = items;
        if (items >= 8LL * grid_req * (region ? kRegions : 1) || total_frames == 0 || px_target <= 65536) break;
        px_target = std::max<int64_t>(65536, px_target / 2);
    }
    // items: largest frames first (their items are the longest), in element order per sequence
    std::vector<size_t> order(p->jobs.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return int64_t(p->jobs[a].W) * p->jobs[a].H * 2 / p->jobs[a].items_per_frame >
               int64_t(p->jobs[b].W) * p->jobs[b].H * 2 / p->jobs[b].items_per_frame;
    });
    std::vector<Item> items;
    items.reserve(static_cast<size_t>(p->n_items));
    for (size_t j : order) {
        const Job& J = p->jobs[j];
        const int hp = J.H / 2;
        for (int64_t k = 0; k < J.n; ++k) {
            for (int part = 0; part < J.items_per_frame; ++part) {
                Item it;
                it.job = static_cast<int32_t>(j);
                it.k = static_cast<int32_t>(k);
                it.rp0 = part * J.item_rp;
                it.nrp = std::min(J.item_rp, hp - it.rp0);
                items.push_back(it);
            }
        }
    }
    p->grid = static_cast<int>(std::min<int64_t>(grid_req, std::max<int64_t>(p->n_items, 1)));
    // device copies (synchronous: plans are built once, then run many times)
    if (p->items_cap < p->n_items) {
        obj_free(p->d_items);
        p->d_items = nullptr;
        p->items_cap = 0;
        void* d = nullptr;
        SCN_CUDA_TRY(obj_alloc(&d, static_cast<size_t>(std::max<int64_t>(p->n_items, 1)) * sizeof(Item)));
        p->d_items = static_cast<Item*>(d);
        p->items_cap = p->n_items;
    }
    if (p->n_items > 0) SCN_CUDA_TRY(obj_upload(p->d_items, items.data(), items.size() * sizeof(Item)));
    SCN_CUDA_TRY(obj_upload(p->d_jobs, p->jobs.data(), p->jobs.size() * sizeof(Job)));
    SCN_CUDA_TRY(obj_finish());  // items and jobs are read from host vectors: done before return
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    return SCN_OK;
}

Launch plan_launch(const scn_plan* p) {
    Launch L{};
    L.jobs = p->d_jobs;
    L.items = p->d_items;
    L.n_items = p->n_items;
    L.queue = reinterpret_cast<uint32_t*>(static_cast<char*>(p->d_block) + 64);
    L.status = static_cast<int*>(p->d_block);
    L.grid = p->grid;
    bool region = true;
    for (const scn_seq* s : p->seqs) region = region && region_frames(s->table->W, s->table->H);
    L.region_items = region ? 1 : 0;
    return L;
}

void free_plan(scn_plan* p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    obj_free(p->d_items);
    obj_free(p->d_jobs);
    obj_free(p->d_block);
    delete p;
}

}  // namespace
}  // namespace scn

using namespace scn;

extern "C" {

scn_status scn_plan_create(scn_seq* const* seqs, int32_t nseq, uint32_t* const* d_hist, uint32_t* const* d_score,
                           uint8_t* const* d_flag, const scn_tune* tune, scn_plan** out) {
    if (!out || nseq < 1 || !seqs || !d_hist || !d_score || !d_flag) return SCN_EINVAL;
    *out = nullptr;
    std::set<const scn_seq*> seen;
    for (int32_t i = 0; i < nseq; ++i) {
        if (!seqs[i] || !seen.insert(seqs[i]).second) return SCN_EINVAL;  // a sequence's scratch serves one job
        if (seqs[i]->n > 0 && (!d_hist[i] || !d_score[i] || !d_flag[i])) return SCN_EINVAL;
        if ((reinterpret_cast<uintptr_t>(d_hist[i]) & 3u) || (reinterpret_cast<uintptr_t>(d_score[i]) & 3u))
            return SCN_EINVAL;
        if (seqs[i]->n > INT32_MAX) return SCN_ERANGE;
    }
    if (tune && (tune->chunk_rows < 0 || (tune->chunk_rows % 2) || tune->grid < 0 || tune->item_kpx < 0))
        return SCN_EINVAL;
    scn_plan* p = new (std::nothrow) scn_plan;
    if (!p) return SCN_ENOMEM;
    p->seqs.assign(seqs, seqs + nseq);
    p->hist.assign(d_hist, d_hist + nseq);
    p->score.assign(d_score, d_score + nseq);
    p->flag.assign(d_flag, d_flag + nseq);
    if (tune) p->tune = *tune;
    void* djobs = nullptr;
    cudaError_t e = obj_alloc(&p->d_block, 256);
    if (e == cudaSuccess) e = obj_zero(p->d_block, 256);
    if (e == cudaSuccess) e = obj_alloc(&djobs, static_cast<size_t>(nseq) * sizeof(Job));
    p->d_jobs = static_cast<Job*>(djobs);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        free_plan(p);
        return SCN_ECUDA;
    }
    const scn_status st = build_items(p);
    if (st != SCN_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return SCN_OK;
}

scn_status scn_plan_destroy(scn_plan* p) {
    if (!p) return SCN_EINVAL;
    free_plan(p);
    return SCN_OK;
}

scn_status scn_plan_set_tune(scn_plan* p, const scn_tune* tune) {
    if (!p || !tune) return SCN_EINVAL;
    if (tune->chunk_rows < 0 || (tune->chunk_rows % 2) || tune->grid < 0 || tune->item_kpx < 0) return SCN_EINVAL;
    p->tune = *tune;
    return build_items(p);
}

scn_status scn_plan_get_tune(const scn_plan* p, scn_tune* tune) {
    if (!p || !tune) return SCN_EINVAL;
    *tune = p->tune;
    return SCN_OK;
}

scn_status scn_plan_info(const scn_plan* p, int64_t* n_items, int64_t* n_frames, int64_t* nv12_bytes, int32_t* grid) {
    if (!p) return SCN_EINVAL;
    int64_t frames = 0, bytes = 0;
    for (const Job& J : p->jobs) {
        frames += J.n;
        bytes += J.n * (static_cast<int64_t>(J.W) * J.H * 3 / 2);
    }
    if (n_items) *n_items = p->n_items;
    if (n_frames) *n_frames = frames;
    if (nv12_bytes) *nv12_bytes = bytes;
    if (grid) *grid = p->grid;
    return SCN_OK;
}

scn_status scn_plan_run(scn_plan* p, void* stream) {
    if (!p) return SCN_EINVAL;
    return launch_hist(plan_launch(p), static_cast<cudaStream_t>(stream));
}

scn_status scn_plan_capture_graph(scn_plan* p, void* stream) {
    if (!p || !stream) return SCN_EINVAL;  // the legacy default stream cannot be captured
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the kernel attribute is set outside the capture
    const scn_status s0 = prepare_hist();
    if (s0 != SCN_OK) return s0;
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    SCN_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const scn_status sl = launch_hist(plan_launch(p), st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (sl != SCN_OK) {
        if (g) cudaGraphDestroy(g);
        return sl;
    }
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SCN_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&p->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        set_cuda_error(ei);
        p->graph = nullptr;
        return SCN_ECUDA;
    }
    return SCN_OK;
}

scn_status scn_plan_replay(scn_plan* p, void* stream) {
    if (!p) return SCN_EINVAL;
    if (!p->graph) return SCN_EINVAL;
    SCN_CUDA_TRY(cudaGraphLaunch(p->graph, static_cast<cudaStream_t>(stream)));
    return SCN_OK;
}

scn_status scn_plan_sync_status(scn_plan* p, void* stream) {
    if (!p) return SCN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    SCN_CUDA_TRY(cudaMemcpyAsync(&h, p->d_block, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCN_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        // a launch that gave up may have left the queue and its sequences'
        // self-clearing scratch part-way: zero them with the status word
        SCN_CUDA_TRY(cudaMemsetAsync(p->d_block, 0, 256, st));
        for (scn_seq* s : p->seqs) SCN_CUDA_TRY(reset_seq_scratch(s, st));
        SCN_CUDA_TRY(cudaStreamSynchronize(st));
        return SCN_ETIMEOUT;
    }
    return SCN_OK;
}

scn_status scn_plan_autotune(scn_plan* p, int32_t reps, void* stream, scn_tune* best, float* best_ms) {
    if (!p || reps < 1) return SCN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int kpx[] = {500, 1000, 2100, 4200, 8400};
    int max_cr = 2;
    for (const Job& J : p->jobs) max_cr = std::max(max_cr, chunk_rows_for(J.W, J.H, 0));
    const int crs[] = {0, std::max(2, (max_cr / 2) & ~1)};
    cudaEvent_t e0, e1;
    SCN_CUDA_TRY(cudaEventCreate(&e0));
    SCN_CUDA_TRY(cudaEventCreate(&e1));
    scn_tune keep = p->tune, win = p->tune;
    float win_ms = 1e30f;
    scn_status rc = SCN_OK;
    for (int cr : crs) {
        for (int kp : kpx) {
            scn_tune t{cr, keep.grid, kp};
            p->tune = t;
            rc = build_items(p);
            if (rc != SCN_OK) break;
            rc = launch_hist(plan_launch(p), st);  // warm
            if (rc != SCN_OK) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == SCN_OK; ++r) rc = launch_hist(plan_launch(p), st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SCN_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= static_cast<float>(reps);
            if (ms < win_ms) {
                win_ms = ms;
                win = t;
            }
        }
        if (rc != SCN_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->tune = rc == SCN_OK ? win : keep;
    const scn_status rb = build_items(p);
    if (rc != SCN_OK) return rc;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return rb;
}

}  // extern "C"
