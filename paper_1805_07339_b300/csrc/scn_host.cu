// Host side of libscn: status text, the synthetic-video shot table, tables,
// sampling and sequences.
//
// Paper anchors: tables with one row per frame (Sec. 3, "Videos as logical
// tables"); sampling by stride, range and index list (Sec. 3.2,
// "Sampling/spacing operations"); the keyframe access pattern (Sec. 5.1.1,
// KEYFRAME).  Storing only some rows of a table mirrors the paper's STRIDED
// storage format (Appendix A.1): sampled rows are materialised, the rest are not.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>

#include "scn_internal.h"

namespace scn {

static thread_local int g_last_cuda_error = 0;

void set_cuda_error(cudaError_t e) { g_last_cuda_error = static_cast<int>(e); }

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return sms;
}

// ---------------------------------------------------------------------------
// SplitMix64 in counter form: output i of the stream seeded with s is
// finalise(s + (i + 1) * gamma)  (Steele, Lea, Flood, OOPSLA 2014).
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

inline uint64_t finalise(uint64_t v) {
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    return v ^ (v >> 31);
}

inline uint64_t draw(uint64_t stream, uint64_t counter) { return finalise(stream + (counter + 1) * kGamma); }

// Shot starts: S-1 distinct boundaries in [1, T-1] (collisions skip to the next
// draw), or geometric lengths 2 + (zero-free 6-bit fields) capped at 300.
bool make_starts(const scn_gen_params& p, std::vector<int64_t>& starts) {
    const uint64_t video = draw(p.master_seed, p.video_id);
    const uint64_t stream = draw(video, 1);
    const int64_t T = p.num_frames;
    starts.clear();
    if (p.shot_mode == 0) {
        const int64_t S = p.num_shots;
        std::set<int64_t> picked;
        uint64_t ctr = 0;
        while (static_cast<int64_t>(picked.size()) < S - 1) {
            picked.insert(1 + static_cast<int64_t>(draw(stream, ctr++) % static_cast<uint64_t>(T - 1)));
        }
        starts.push_back(0);
        starts.insert(starts.end(), picked.begin(), picked.end());
        return true;
    }
    uint64_t word = 0, wctr = 0;
    int left = 0;  // 6-bit fields left in word
    int64_t at = 0;
    while (at < T) {
        starts.push_back(at);
        int64_t len = 2;
        while (len < 300) {
            if (left == 0) {
                word = draw(stream, wctr++);
                left = 10;
            }
            const uint64_t field = word & 63u;
            word >>= 6;
            --left;
            if (field == 0) break;
            ++len;
        }
        at += len;
    }
    return true;
}

inline int64_t dist(int64_t a, int64_t b) { return a < b ? b - a : a - b; }

}  // namespace

bool build_shots(const scn_gen_params& p, std::vector<scn_shot>& out) {
    std::vector<int64_t> starts;
    if (!make_starts(p, starts)) return false;
    const uint64_t colours = draw(draw(p.master_seed, p.video_id), 3);
    uint64_t ctr = 0;
    out.assign(starts.size(), scn_shot{});
    for (size_t i = 0; i < starts.size(); ++i) {
        int64_t b[3];
        for (;;) {
            b[0] = 16 + static_cast<int64_t>(draw(colours, ctr) % 220u);
            b[1] = 16 + static_cast<int64_t>(draw(colours, ctr + 1) % 225u);
            b[2] = 16 + static_cast<int64_t>(draw(colours, ctr + 2) % 225u);
            ctr += 3;
            if (i == 0) break;
            const scn_shot& prev = out[i - 1];
            const bool close_y = dist(b[0], prev.base[0]) < 48;
            const bool close_uv = dist(b[1], prev.base[1]) + dist(b[2], prev.base[2]) < 64;
            if (!(close_y && close_uv)) break;
        }
        scn_shot& s = out[i];
        s.start = starts[i];
        for (int pl = 0; pl < 3; ++pl) s.base[pl] = static_cast<int32_t>(b[pl]);
        for (int pl = 0; pl < 3; ++pl) {
            s.gx[pl] = static_cast<int32_t>(draw(colours, ctr++) % 65u) - 32;
            s.gy[pl] = static_cast<int32_t>(draw(colours, ctr++) % 65u) - 32;
        }
    }
    return true;
}

bool gen_params_ok(const scn_gen_params* p) {
    if (!p) return false;
    if (p->width < 16 || p->height < 2 || (p->width % 16) || (p->height % 2)) return false;
    if (p->num_frames < 1) return false;
    if (p->shot_mode == 0) {
        if (p->num_shots < 1 || p->num_shots > p->num_frames) return false;
    } else if (p->shot_mode != 1) {
        return false;
    }
    return true;
}

}  // namespace scn

using namespace scn;

namespace scn {
cudaError_t reset_seq_scratch(scn_seq* s, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(static_cast<char*>(s->d_block) + s->scratch_off, 0, s->scratch_bytes, st);
    if (e == cudaSuccess) e = reset_gate_workspace(s, st);
    return e;
}
}  // namespace scn

extern "C" {

const char* scn_status_str(scn_status s) {
    switch (s) {
        case SCN_OK: return "ok";
        case SCN_EINVAL: return "invalid argument";
        case SCN_ERANGE: return "index or size out of range";
        case SCN_ENOMEM: return "out of memory";
        case SCN_ECUDA: return "CUDA runtime error";
        case SCN_ETIMEOUT: return "bounded device wait timed out";
        case SCN_EUNSUPPORTED: return "unsupported device or request";
    }
    return "unknown status";
}

int scn_last_cuda_error(void) { return g_last_cuda_error; }

const char* scn_version(void) { return "scn 0.1 (sm_103a)"; }

int scn_device_sm_count(void) { return device_sm_count(); }

// ---------------------------------------------------------------------------
// video (generator shot table)
// ---------------------------------------------------------------------------
scn_status scn_gen_shots(const scn_gen_params* params, scn_shot* h_out, int64_t cap, int64_t* n) {
    if (!n || cap < 0 || (cap > 0 && !h_out) || !gen_params_ok(params)) return SCN_EINVAL;
    std::vector<scn_shot> shots;
    if (!build_shots(*params, shots)) return SCN_EINVAL;
    *n = static_cast<int64_t>(shots.size());
    const int64_t m = std::min<int64_t>(cap, *n);
    if (m > 0) std::memcpy(h_out, shots.data(), static_cast<size_t>(m) * sizeof(scn_shot));
    return SCN_OK;
}

scn_status scn_video_create(const scn_gen_params* params, scn_video** out) {
    if (!out || !gen_params_ok(params)) return SCN_EINVAL;
    *out = nullptr;
    scn_video* v = new (std::nothrow) scn_video;
    if (!v) return SCN_ENOMEM;
    v->p = *params;
    if (!build_shots(v->p, v->shots)) {
        delete v;
        return SCN_EINVAL;
    }
    const size_t bytes = v->shots.size() * sizeof(scn_shot);
    void* d = nullptr;
    cudaError_t e = obj_alloc(&d, bytes);
    v->d_shots = static_cast<scn_shot*>(d);
    if (e == cudaSuccess) e = obj_upload(v->d_shots, v->shots.data(), bytes);
    if (e == cudaSuccess) e = obj_finish();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        obj_free(v->d_shots);
        delete v;
        return e == cudaErrorMemoryAllocation ? SCN_ENOMEM : SCN_ECUDA;
    }
    *out = v;
    return SCN_OK;
}

scn_status scn_video_destroy(scn_video* v) {
    if (!v) return SCN_EINVAL;
    obj_free(v->d_shots);
    delete v;
    return SCN_OK;
}

scn_status scn_video_shots(const scn_video* v, scn_shot* h_out, int64_t cap, int64_t* n) {
    if (!v || !n || cap < 0 || (cap > 0 && !h_out)) return SCN_EINVAL;
    *n = static_cast<int64_t>(v->shots.size());
    const int64_t m = std::min<int64_t>(cap, *n);
    if (m > 0) std::memcpy(h_out, v->shots.data(), static_cast<size_t>(m) * sizeof(scn_shot));
    return SCN_OK;
}

scn_status scn_video_keyframes(const scn_video* v, int64_t* h_out, int64_t cap, int64_t* n) {
    if (!v || !n || cap < 0 || (cap > 0 && !h_out)) return SCN_EINVAL;
    std::set<int64_t> k;
    for (int64_t f = 0; f < v->p.num_frames; f += 104) k.insert(f);
    for (const scn_shot& s : v->shots) k.insert(s.start);
    *n = static_cast<int64_t>(k.size());
    int64_t i = 0;
    for (int64_t f : k) {
        if (i >= cap) break;
        h_out[i++] = f;
    }
    return SCN_OK;
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
scn_status scn_table_create(const scn_table_desc* d, scn_table** out) {
    if (!d || !out) return SCN_EINVAL;
    *out = nullptr;
    if (d->width < 16 || d->height < 2 || (d->width % 16) || (d->height % 2)) return SCN_EINVAL;
    if (d->num_frames < 0) return SCN_EINVAL;
    const int64_t fb = static_cast<int64_t>(d->width) * d->height * 3 / 2;
    if (d->frame_stride < fb || (d->frame_stride % 16)) return SCN_EINVAL;
    if (!d->d_nv12 || !aligned16(d->d_nv12)) return SCN_EINVAL;
    if (d->h_rows && d->num_rows < 0) return SCN_EINVAL;
    if (d->h_keyframes && d->num_keyframes < 0) return SCN_EINVAL;
    scn_table* t = new (std::nothrow) scn_table;
    if (!t) return SCN_ENOMEM;
    t->W = d->width;
    t->H = d->height;
    t->num_frames = d->num_frames;
    t->frame_stride = d->frame_stride;
    t->d_nv12 = d->d_nv12;
    if (d->h_rows) {
        t->rows.assign(d->h_rows, d->h_rows + d->num_rows);
        for (size_t i = 0; i < t->rows.size(); ++i) {
            const bool bad = t->rows[i] < 0 || t->rows[i] >= d->num_frames || (i && t->rows[i] <= t->rows[i - 1]);
            if (bad) {
                delete t;
                return SCN_EINVAL;
            }
        }
    }
    if (d->h_keyframes) {
        std::set<int64_t> k(d->h_keyframes, d->h_keyframes + d->num_keyframes);
        for (int64_t f : k) {
            if (f < 0 || f >= d->num_frames) {
                delete t;
                return SCN_EINVAL;
            }
        }
        t->keyframes.assign(k.begin(), k.end());
    }
    *out = t;
    return SCN_OK;
}

scn_status scn_table_destroy(scn_table* t) {
    if (!t) return SCN_EINVAL;
    delete t;
    return SCN_OK;
}

// ---------------------------------------------------------------------------
// sampling
// ---------------------------------------------------------------------------
static scn_status select_frames(const scn_table* t, const scn_sample_spec* sp, std::vector<int64_t>& f) {
    f.clear();
    switch (sp->kind) {
        case SCN_STRIDE:
        case SCN_RANGE: {
            const int64_t step = sp->kind == SCN_RANGE ? 1 : sp->step;
            if (step < 1) return SCN_EINVAL;
            if (sp->start < 0 || sp->stop > t->num_frames) return SCN_ERANGE;
            for (int64_t i = sp->start; i < sp->stop; i += step) f.push_back(i);
            return SCN_OK;
        }
        case SCN_GATHER: {
            if (sp->n < 0 || (sp->n > 0 && !sp->h_indices)) return SCN_EINVAL;
            for (int64_t i = 0; i < sp->n; ++i) {
                if (sp->h_indices[i] < 0 || sp->h_indices[i] >= t->num_frames) return SCN_ERANGE;
            }
            f.assign(sp->h_indices, sp->h_indices + sp->n);
            return SCN_OK;
        }
        case SCN_KEYFRAME:
            f = t->keyframes;
            return SCN_OK;
        default:
            return SCN_EINVAL;
    }
}

// storage slot of each selected frame (dense tables: the frame number itself)
static scn_status slots_of(const scn_table* t, const std::vector<int64_t>& f, std::vector<int32_t>& slot) {
    slot.resize(f.size());
    for (size_t i = 0; i < f.size(); ++i) {
        int64_t s = f[i];
        if (!t->rows.empty()) {
            auto it = std::lower_bound(t->rows.begin(), t->rows.end(), f[i]);
            if (it == t->rows.end() || *it != f[i]) return SCN_ERANGE;
            s = it - t->rows.begin();
        }
        if (s > INT32_MAX) return SCN_ERANGE;
        slot[i] = static_cast<int32_t>(s);
    }
    return SCN_OK;
}

scn_status scn_sample_indices(const scn_table* t, const scn_sample_spec* spec, int64_t* h_out, int64_t cap,
                              int64_t* n) {
    if (!t || !spec || !n || cap < 0 || (cap > 0 && !h_out)) return SCN_EINVAL;
    std::vector<int64_t> f;
    scn_status st = select_frames(t, spec, f);
    if (st != SCN_OK) return st;
    std::vector<int32_t> slot;
    st = slots_of(t, f, slot);
    if (st != SCN_OK) return st;
    *n = static_cast<int64_t>(f.size());
    const int64_t m = std::min<int64_t>(cap, *n);
    for (int64_t i = 0; i < m; ++i) h_out[i] = f[i];
    return SCN_OK;
}

scn_status scn_sample(const scn_table* t, const scn_sample_spec* spec, scn_seq** out) {
    if (!t || !spec || !out) return SCN_EINVAL;
    *out = nullptr;
    std::vector<int64_t> f;
    scn_status st = select_frames(t, spec, f);
    if (st != SCN_OK) return st;
    std::vector<int32_t> slot;
    st = slots_of(t, f, slot);
    if (st != SCN_OK) return st;
    scn_seq* s = new (std::nothrow) scn_seq;
    if (!s) return SCN_ENOMEM;
    s->table = t;
    s->n = static_cast<int64_t>(f.size());
    s->frames = std::move(f);
    const size_t n = static_cast<size_t>(std::max<int64_t>(s->n, 1));
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_slot = up(n * 4), b_done = up(n * 4), b_pair = up(n * 4);
    const size_t b_part = up(n * 48 * 4), b_stat = 256;
    const size_t total = b_slot + b_done + b_pair + b_part + b_stat;
    cudaError_t e = obj_alloc(&s->d_block, total);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        delete s;
        return e == cudaErrorMemoryAllocation ? SCN_ENOMEM : SCN_ECUDA;
    }
    char* p = static_cast<char*>(s->d_block);
    s->d_slot = reinterpret_cast<int32_t*>(p);
    s->d_done = reinterpret_cast<uint32_t*>(p + b_slot);
    s->d_pair = reinterpret_cast<uint32_t*>(p + b_slot + b_done);
    s->d_partial = reinterpret_cast<uint32_t*>(p + b_slot + b_done + b_pair);
    s->d_status = reinterpret_cast<int*>(p + b_slot + b_done + b_pair + b_part);
    s->d_queue = reinterpret_cast<uint32_t*>(p + b_slot + b_done + b_pair + b_part + 64);
    s->scratch_off = b_slot;
    s->scratch_bytes = total - b_slot;
    e = obj_zero(s->d_block, total);
    if (e == cudaSuccess && s->n > 0) e = obj_upload(s->d_slot, slot.data(), slot.size() * 4);
    if (e == cudaSuccess) e = obj_finish();  // the slot list is read from host memory: done before return
    if (e != cudaSuccess) {
        set_cuda_error(e);
        obj_free(s->d_block);
        delete s;
        return SCN_ECUDA;
    }
    *out = s;
    return SCN_OK;
}

scn_status scn_seq_length(const scn_seq* s, int64_t* n) {
    if (!s || !n) return SCN_EINVAL;
    *n = s->n;
    return SCN_OK;
}

scn_status scn_seq_destroy(scn_seq* s) {
    if (!s) return SCN_EINVAL;
    free_gate_workspace(s);
    free_space_workspace(s);
    obj_free(s->d_block);
    delete s;
    return SCN_OK;
}

scn_status scn_seq_sync_status(scn_seq* s, void* stream) {
    if (!s) return SCN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    SCN_CUDA_TRY(cudaMemcpyAsync(&h, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCN_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        // a launch that gave up may have left its self-clearing scratch part-way
        // (partial histograms, counters, the queue): zero it with the status word
        SCN_CUDA_TRY(reset_seq_scratch(s, st));
        SCN_CUDA_TRY(cudaStreamSynchronize(st));
        return SCN_ETIMEOUT;
    }
    return SCN_OK;
}

scn_status scn_seq_set_wait_test(scn_seq* s, uint64_t wait_limit_ns, int32_t withhold_after) {
    if (!s) return SCN_EINVAL;
    if (wait_limit_ns != 0 && (wait_limit_ns < 100000ull || wait_limit_ns > 10000000000ull)) return SCN_EINVAL;
    s->test_wait_ns = wait_limit_ns;
    s->test_withhold = withhold_after < 0 ? -1 : withhold_after;
    return SCN_OK;
}

scn_status scn_seq_set_tune(scn_seq* s, const scn_tune* tune) {
    if (!s || !tune) return SCN_EINVAL;
    if (tune->chunk_rows < 0 || (tune->chunk_rows % 2)) return SCN_EINVAL;
    if (tune->grid < 0 || tune->item_kpx < 0) return SCN_EINVAL;
    s->tune = *tune;
    return SCN_OK;
}

scn_status scn_seq_get_tune(const scn_seq* s, scn_tune* tune) {
    if (!s || !tune) return SCN_EINVAL;
    const HistShape sh = resolve_hist_shape(s);
    tune->chunk_rows = sh.chunk_rows;
    tune->grid = sh.grid;
    tune->item_kpx = sh.rp_per_cta > 0 ? 0
                                       : static_cast<int32_t>((static_cast<int64_t>(sh.item_rp) * 2 * s->table->W + 999) / 1000);
    return SCN_OK;
}

}  // extern "C"
