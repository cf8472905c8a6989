/*
 * orc.c - the CPU oracle for the sampled-frame convert / histogram / shot-score /
 * resize path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, the smoke check in __graft_entry__.py and the CPU
 * baseline leg of bench.py use it.  It shares no source with the CUDA library.
 *
 * Every routine is the plain definition, written for readability, not speed:
 * one pixel at a time, fp64 where floating point appears.
 *
 * Sources.  The paper (Scanner, Poms et al., ACM TOG 37(4) 2018) defines the
 * model - videos as tables of frames (Sec. 3, "Videos as logical tables"),
 * sampling by stride / range / index list (Sec. 3.2, "Sampling/spacing
 * operations"), a two-element stencil over consecutive elements (Sec. 3.2,
 * "Stencil operations"), a per-frame colour histogram (Sec. 5.1.2, HIST) and
 * shot boundaries from histogram differences (Sec. 5.2, data mining).  It fixes
 * no pixel arithmetic; the constants below are the readings stated in the
 * repository's design notes:
 *   - generator: SplitMix64 counter stream (Steele, Lea and Flood, OOPSLA 2014),
 *     shots with a base colour, a drifting linear ramp and Irwin-Hall noise;
 *   - BT.601 limited-range 8-bit conversion with the x256 rounded coefficients
 *     298 / 409 / 100 / 208 / 516;
 *   - 16 bins per channel, bin = value >> 4;
 *   - L1 distance of consecutive histograms, flag when 2*score > W*H;
 *   - bilinear resize with half-pixel centres (align_corners = false, no
 *     antialias) followed by (v/255 - mean)/std.
 *
 * Parity pins: see tests/test_oracle_*.py (SplitMix64 published vectors, BT.601
 * colour bars, float BT.601 within one level, exact Irwin-Hall pmf, library
 * bilinear interpolation, brute-force histograms, finite differences).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden gamma  */
/* and each output is the mix64 finaliser of the state.  Counter form:       */
/* the i-th output (0-based) of a stream seeded with s is mix(s + (i+1)*G).  */
/* ------------------------------------------------------------------------ */
static const uint64_t ORC_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t orc_mix64(uint64_t z) {
    z = z ^ (z >> 30);
    z = z * 0xBF58476D1CE4E5B9ULL;
    z = z ^ (z >> 27);
    z = z * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return z;
}

uint64_t orc_sm(uint64_t seed, uint64_t i) {
    return orc_mix64(seed + (i + 1) * ORC_GAMMA);
}

/* floor division for a positive divisor */
static int64_t orc_floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static int64_t orc_clampi(int64_t v, int64_t lo, int64_t hi) {
    if (v < lo) return lo;
    if (v > hi) return hi;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Generator: shot table                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t master_seed;
    uint64_t video_id;
    int32_t width, height;
    int64_t num_frames;
    int32_t num_shots;   /* uniform mode: number of shots S (>= 1) */
    int32_t shot_mode;   /* 0: S-1 uniform boundaries, 1: geometric lengths */
} orc_gen_params;

typedef struct {
    int64_t start;       /* first frame of the shot */
    int32_t base[3];     /* Y, U, V base level */
    int32_t gx[3];       /* horizontal ramp amplitude per plane */
    int32_t gy[3];       /* vertical ramp amplitude per plane */
} orc_shot;

static uint64_t orc_video_seed(const orc_gen_params* p) {
    return orc_sm(p->master_seed, p->video_id);
}

static int orc_cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Shot starts.  Returns the number of shots, or -1 if cap is too small or the
 * request is impossible. */
static int64_t orc_shot_starts(const orc_gen_params* p, int64_t* starts, int64_t cap) {
    uint64_t s_v = orc_video_seed(p);
    uint64_t s_shot = orc_sm(s_v, 1);
    int64_t T = p->num_frames;
    if (T < 1) return -1;
    if (p->shot_mode == 0) {
        int64_t S = p->num_shots;
        if (S < 1 || S > T || S > cap) return -1;
        starts[0] = 0;
        int64_t have = 0;               /* boundaries drawn so far */
        uint64_t j = 0;
        while (have < S - 1) {
            int64_t b = 1 + (int64_t)(orc_sm(s_shot, j) % (uint64_t)(T - 1));
            j++;
            int dup = 0;
            for (int64_t k = 0; k < have; k++) {
                if (starts[1 + k] == b) { dup = 1; break; }
            }
            if (!dup) { starts[1 + have] = b; have++; }
        }
        qsort(starts + 1, (size_t)(S - 1), sizeof(int64_t), orc_cmp_i64);
        return S;
    }
    /* geometric: L = 2 + failures before the first zero 6-bit field, at most 300 */
    int64_t n = 0, pos = 0;
    uint64_t word_index = 0;
    int field = 10;                     /* forces a fresh word on first use */
    uint64_t word = 0;
    while (pos < T) {
        if (n >= cap) return -1;
        starts[n++] = pos;
        int64_t failures = 0;
        for (;;) {
            if (2 + failures >= 300) break;
            if (field == 10) { word = orc_sm(s_shot, word_index); word_index++; field = 0; }
            uint64_t f = (word >> (6 * field)) & 63u;
            field++;
            if (f == 0) break;
            failures++;
        }
        pos += 2 + failures;
    }
    return n;
}

static int64_t orc_absdiff(int64_t a, int64_t b) { return a > b ? a - b : b - a; }

/* Full shot table: starts plus per-shot colours and ramps drawn in order from
 * the stream SM(s_v, 3). */
int64_t orc_gen_shots(const orc_gen_params* p, orc_shot* out, int64_t cap) {
    int64_t* starts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    if (!starts) return -1;
    int64_t n = orc_shot_starts(p, starts, cap);
    if (n < 0) { free(starts); return -1; }
    uint64_t s_col = orc_sm(orc_video_seed(p), 3);
    uint64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t Yb, Ub, Vb;
        for (;;) {
            Yb = 16 + (int64_t)(orc_sm(s_col, c++) % 220u);
            Ub = 16 + (int64_t)(orc_sm(s_col, c++) % 225u);
            Vb = 16 + (int64_t)(orc_sm(s_col, c++) % 225u);
            if (i == 0) break;
            int64_t dy = orc_absdiff(Yb, out[i - 1].base[0]);
            int64_t duv = orc_absdiff(Ub, out[i - 1].base[1]) + orc_absdiff(Vb, out[i - 1].base[2]);
            if (!(dy < 48 && duv < 64)) break;   /* too close to the previous shot: redraw */
        }
        out[i].start = starts[i];
        out[i].base[0] = (int32_t)Yb;
        out[i].base[1] = (int32_t)Ub;
        out[i].base[2] = (int32_t)Vb;
        for (int pl = 0; pl < 3; pl++) {
            out[i].gx[pl] = (int32_t)(orc_sm(s_col, c++) % 65u) - 32;
            out[i].gy[pl] = (int32_t)(orc_sm(s_col, c++) % 65u) - 32;
        }
    }
    free(starts);
    return n;
}

/* Irwin-Hall noise for sample q: 12 uniform bytes (8 of w0, the low 4 of w1),
 * centred on 1530 and scaled by 1/32 with a rounding offset: sigma = 8. */
int32_t orc_noise(uint64_t s_pix, uint64_t q) {
    uint64_t w0 = orc_sm(s_pix, 2 * q);
    uint64_t w1 = orc_sm(s_pix, 2 * q + 1);
    int64_t S = 0;
    for (int b = 0; b < 8; b++) S += (int64_t)((w0 >> (8 * b)) & 255u);
    for (int b = 0; b < 4; b++) S += (int64_t)((w1 >> (8 * b)) & 255u);
    return (int32_t)orc_floordiv(S - 1530 + 16, 32);
}

/* One NV12 frame: Y plane H x W, then H/2 rows of interleaved U,V.  out must
 * hold W*H*3/2 bytes. */
void orc_gen_frame(const orc_gen_params* p, const orc_shot* shots, int64_t nshots,
                   int64_t frame, uint8_t* out) {
    const int64_t W = p->width, H = p->height;
    uint64_t s_pix = orc_sm(orc_video_seed(p), 2);
    /* the shot containing this frame: the last one whose start <= frame */
    int64_t si = 0;
    for (int64_t i = 0; i < nshots; i++) {
        if (shots[i].start <= frame) si = i;
    }
    const orc_shot* sh = &shots[si];
    int64_t dt = frame - sh->start;
    for (int pl = 0; pl < 3; pl++) {
        int64_t Wp = (pl == 0) ? W : W / 2;
        int64_t Hp = (pl == 0) ? H : H / 2;
        int64_t hi = (pl == 0) ? 235 : 240;
        for (int64_t yp = 0; yp < Hp; yp++) {
            for (int64_t xp = 0; xp < Wp; xp++) {
                int64_t x = (pl == 0) ? xp : 2 * xp;   /* luma coordinates */
                int64_t y = (pl == 0) ? yp : 2 * yp;
                uint64_t q = (uint64_t)(((frame * 3 + pl) * Hp + yp) * Wp + xp);
                int64_t v = sh->base[pl]
                          + orc_floordiv((int64_t)sh->gx[pl] * (x - dt), W)
                          + orc_floordiv((int64_t)sh->gy[pl] * y, H)
                          + orc_noise(s_pix, q);
                v = orc_clampi(v, 16, hi);
                if (pl == 0) {
                    out[yp * W + xp] = (uint8_t)v;
                } else {
                    /* U at even byte, V at odd byte of the UV row */
                    out[W * H + yp * W + 2 * xp + (pl - 1)] = (uint8_t)v;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* BT.601 limited range -> RGB, 8-bit fixed point                            */
/* ------------------------------------------------------------------------ */
void orc_yuv_to_rgb(int32_t Y, int32_t U, int32_t V, int32_t rgb[3]) {
    int64_t C = Y - 16, D = U - 128, E = V - 128;
    rgb[0] = (int32_t)orc_clampi(orc_floordiv(298 * C + 409 * E + 128, 256), 0, 255);
    rgb[1] = (int32_t)orc_clampi(orc_floordiv(298 * C - 100 * D - 208 * E + 128, 256), 0, 255);
    rgb[2] = (int32_t)orc_clampi(orc_floordiv(298 * C + 516 * D + 128, 256), 0, 255);
}

/* Convert n packed (Y, U, V) byte triples to (R, G, B) byte triples. */
void orc_yuv_to_rgb_array(const uint8_t* yuv, int64_t n, uint8_t* rgb) {
    for (int64_t i = 0; i < n; i++) {
        int32_t px[3];
        orc_yuv_to_rgb(yuv[3 * i], yuv[3 * i + 1], yuv[3 * i + 2], px);
        for (int c = 0; c < 3; c++) rgb[3 * i + c] = (uint8_t)px[c];
    }
}

/* RGB of pixel (x, y) of an NV12 frame; chroma is the nearest sample (x>>1, y>>1). */
static void orc_pixel_rgb(const uint8_t* f, int64_t W, int64_t H, int64_t x, int64_t y, int32_t rgb[3]) {
    int32_t Y = f[y * W + x];
    const uint8_t* uv = f + W * H + (y / 2) * W + 2 * (x / 2);
    orc_yuv_to_rgb(Y, uv[0], uv[1], rgb);
}

/* hist[c*16 + b] = number of pixels whose channel c value v has v >> 4 == b */
void orc_hist_frame(const uint8_t* f, int32_t W, int32_t H, uint32_t hist[48]) {
    for (int i = 0; i < 48; i++) hist[i] = 0;
    for (int64_t y = 0; y < H; y++) {
        for (int64_t x = 0; x < W; x++) {
            int32_t rgb[3];
            orc_pixel_rgb(f, W, H, x, y, rgb);
            for (int c = 0; c < 3; c++) hist[c * 16 + rgb[c] / 16] += 1;
        }
    }
}

/* score[0] = 0; score[k] = sum over the 48 bins of |hist[k] - hist[k-1]|;
 * flag[k] = 2*score[k] > pixel_count (score > half the pixel count). */
void orc_scores(const uint32_t* hist, int64_t n, int64_t pixel_count, uint32_t* score, uint8_t* flag) {
    for (int64_t k = 0; k < n; k++) {
        int64_t s = 0;
        if (k > 0) {
            for (int i = 0; i < 48; i++) {
                s += orc_absdiff((int64_t)hist[k * 48 + i], (int64_t)hist[(k - 1) * 48 + i]);
            }
        }
        score[k] = (uint32_t)s;
        flag[k] = (uint8_t)(2 * s > pixel_count ? 1 : 0);
    }
}

/* ------------------------------------------------------------------------ */
/* Bilinear resize (half-pixel centres, source index clamped at 0, upper     */
/* neighbour clamped to the last row/column) + per-channel normalisation.   */
/* out is [3][oh][ow] fp64.                                                  */
/* ------------------------------------------------------------------------ */
void orc_resize_norm_frame(const uint8_t* f, int32_t W, int32_t H, int32_t oh, int32_t ow,
                           const double mean[3], const double stdv[3], double* out) {
    /* the converted full-resolution image first, as three uint8 planes */
    uint8_t* rgb = (uint8_t*)malloc((size_t)W * (size_t)H * 3);
    if (!rgb) return;
    for (int64_t y = 0; y < H; y++) {
        for (int64_t x = 0; x < W; x++) {
            int32_t px[3];
            orc_pixel_rgb(f, W, H, x, y, px);
            for (int c = 0; c < 3; c++) rgb[(c * (int64_t)H + y) * W + x] = (uint8_t)px[c];
        }
    }
    double sy_scale = (double)H / (double)oh;
    double sx_scale = (double)W / (double)ow;
    for (int c = 0; c < 3; c++) {
        const uint8_t* P = rgb + (int64_t)c * H * W;
        for (int64_t oy = 0; oy < oh; oy++) {
            double sy = ((double)oy + 0.5) * sy_scale - 0.5;
            if (sy < 0) sy = 0;
            int64_t y0 = (int64_t)floor(sy);
            int64_t y1 = y0 + 1 < H ? y0 + 1 : H - 1;
            double ly = sy - (double)y0;
            for (int64_t ox = 0; ox < ow; ox++) {
                double sx = ((double)ox + 0.5) * sx_scale - 0.5;
                if (sx < 0) sx = 0;
                int64_t x0 = (int64_t)floor(sx);
                int64_t x1 = x0 + 1 < W ? x0 + 1 : W - 1;
                double lx = sx - (double)x0;
                double v = (1 - ly) * ((1 - lx) * P[y0 * W + x0] + lx * P[y0 * W + x1])
                         + ly * ((1 - lx) * P[y1 * W + x0] + lx * P[y1 * W + x1]);
                out[((int64_t)c * oh + oy) * ow + ox] = (v / 255.0 - mean[c]) / stdv[c];
            }
        }
    }
    free(rgb);
}

/* thumb[r][c] = Y[s*r][s*c], s = W/64 (= H/36), r < 36, c < 64 */
void orc_thumb_frame(const uint8_t* f, int32_t W, int32_t H, uint8_t* thumb) {
    int64_t s = W / 64;
    (void)H;
    for (int64_t r = 0; r < 36; r++)
        for (int64_t c = 0; c < 64; c++)
            thumb[r * 64 + c] = f[(s * r) * W + s * c];
}

/* Coarse YUV thumbnails: every sixth row and every second column of the luma
 * thumbnail grid, and the chroma sample under each of those pixels.
 * yuv[0][r][c] = Y at luma pixel (2 s c, 6 s r); yuv[1][r][c] and yuv[2][r][c]
 * = U and V of chroma sample (s c, 3 s r), the one that pixel uses; r < 6,
 * c < 32.  In the NV12 chroma plane (H/2 rows of W bytes, U and V interleaved)
 * that sample's U is byte 2 s c of row 3 s r and its V the next byte. */
void orc_thumb_yuv_frame(const uint8_t* f, int32_t W, int32_t H, uint8_t* yuv) {
    int64_t s = W / 64;
    const uint8_t* plane = f + (int64_t)W * H;
    for (int64_t r = 0; r < 6; r++)
        for (int64_t c = 0; c < 32; c++) {
            yuv[(0 * 6 + r) * 32 + c] = f[(6 * s * r) * W + 2 * s * c];
            yuv[(1 * 6 + r) * 32 + c] = plane[(3 * s * r) * W + 2 * (s * c)];
            yuv[(2 * 6 + r) * 32 + c] = plane[(3 * s * r) * W + 2 * (s * c) + 1];
        }
}

/* The luma thumbnail-difference gate between frames k-1 and k: the mean
 * absolute difference of their 36 x 64 luma thumbnails. */
double orc_thumb_diff(const uint8_t* ta, const uint8_t* tb) {
    int64_t sy = 0;
    for (int64_t i = 0; i < 2304; i++) sy += labs((long)ta[i] - (long)tb[i]);
    return (double)sy / 2304.0;
}

/* The luma + chroma gate: over two coarse YUV thumbnails, the mean absolute
 * difference of the Y samples plus that of the U samples plus that of the V
 * samples (192 each). */
double orc_thumb_diff_yuv(const uint8_t* ya, const uint8_t* yb) {
    double d = 0.0;
    for (int64_t p = 0; p < 3; p++) {
        int64_t sp = 0;
        for (int64_t i = 0; i < 192; i++) sp += labs((long)ya[p * 192 + i] - (long)yb[p * 192 + i]);
        d += (double)sp / 192.0;
    }
    return d;
}

/* ------------------------------------------------------------------------ */
/* Batch wrappers (frames split statically over plain pthreads).  These only */
/* loop the per-frame definitions above.                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint8_t* frames; int64_t frame_bytes; int32_t W, H;
    const int64_t* idx; int64_t lo, hi; uint32_t* hist;
} orc_hist_job;

static void* orc_hist_worker(void* arg) {
    orc_hist_job* j = (orc_hist_job*)arg;
    for (int64_t k = j->lo; k < j->hi; k++) {
        int64_t fi = j->idx ? j->idx[k] : k;
        orc_hist_frame(j->frames + fi * j->frame_bytes, j->W, j->H, j->hist + k * 48);
    }
    return NULL;
}

/* hist[k] of frame idx[k] (or frame k when idx is NULL) of a contiguous frame
 * array; nthreads >= 1. */
void orc_hist_batch(const uint8_t* frames, int64_t frame_bytes, int32_t W, int32_t H,
                    const int64_t* idx, int64_t n, int32_t nthreads, uint32_t* hist) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    orc_hist_job jobs[256];
    int64_t per = (n + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        int64_t lo = t * per, hi = lo + per;
        if (hi > n) hi = n;
        if (lo >= hi) break;
        jobs[t] = (orc_hist_job){frames, frame_bytes, W, H, idx, lo, hi, hist};
        if (nthreads == 1) { orc_hist_worker(&jobs[t]); continue; }
        pthread_create(&th[t], NULL, orc_hist_worker, &jobs[t]);
        started = t + 1;
    }
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
}

typedef struct {
    const orc_gen_params* p; const orc_shot* shots; int64_t nshots;
    const int64_t* frames; int64_t lo, hi; uint8_t* out; int64_t frame_bytes;
} orc_gen_job;

static void* orc_gen_worker(void* arg) {
    orc_gen_job* j = (orc_gen_job*)arg;
    for (int64_t k = j->lo; k < j->hi; k++)
        orc_gen_frame(j->p, j->shots, j->nshots, j->frames[k], j->out + k * j->frame_bytes);
    return NULL;
}

/* Generate frames[k] into out + k*frame_bytes for k < n. */
void orc_gen_batch(const orc_gen_params* p, const orc_shot* shots, int64_t nshots,
                   const int64_t* frames, int64_t n, int64_t frame_bytes, int32_t nthreads,
                   uint8_t* out) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    orc_gen_job jobs[256];
    int64_t per = (n + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        int64_t lo = t * per, hi = lo + per;
        if (hi > n) hi = n;
        if (lo >= hi) break;
        jobs[t] = (orc_gen_job){p, shots, nshots, frames, lo, hi, out, frame_bytes};
        if (nthreads == 1) { orc_gen_worker(&jobs[t]); continue; }
        pthread_create(&th[t], NULL, orc_gen_worker, &jobs[t]);
        started = t + 1;
    }
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
}
