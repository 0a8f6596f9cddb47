/*
 * bm_oracle.c -- plain CPU brute-force block matcher.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it computes (Self-Convolution paper, arXiv 2006.13714):
 *
 *   For every reference patch X_r (top-left corner r on the reference grid)
 *   and every candidate patch X_j whose top-left corner lies in the search
 *   window Omega_r, the squared Euclidean distance
 *
 *       d_E(X_j, X_r) = || X_j - X_r ||_F^2                    (§III-A, Eq. equ:bm;
 *                                                             §III-E, Eq. equ:bmMetric_app)
 *
 *   summed over all channels of a 3-D patch (§IV, 2-D Self-Convolution
 *   with the channel summation S(.) of Eq. equ:self-convMM), then the K
 *   candidates of smallest distance (the arg-min over |S_r| <= K of Eq.
 *   equ:bm).  The window restriction is the X_{Omega_i} generalisation of
 *   the footnote to Eq. eq:unifySelfConv (§III-B).
 *
 * Readings where the paper is silent (stated once here, used everywhere):
 *   - window  = W_s x W_s candidate top-left offsets centred on r,
 *               dy, dx in [-h, h], h = (W_s - 1) / 2, W_s odd;
 *   - borders = the window is clipped to the valid top-left grid
 *               [0, H-p] x [0, W-p]; no padding, no shifting;
 *   - refs    = {(s*a, s*b)} inside that grid, row-major; count per axis
 *               floor((H-p)/s) + 1;
 *   - ties    = (distance ascending, row-major offset y*W + x ascending);
 *   - |Omega_r| < K: the tail is idx = -1, dist = sentinel.
 *
 * Arithmetic: int64 for uint8 input (exact), IEEE double for float32 input.
 * Image layout: H x W x C, channels innermost, row-major.
 *
 * Two evaluations of the same distance are provided:
 *   bmo_match_*      -- the definition, sum of (X_r - X_j)^2 written out;
 *   bmo_selfconv_*   -- Lemma 2 (§III-B): ||X_j||^2 + ||X_r||^2 - 2 C_r(j),
 *                       with ||X_j||^2 a box sum of the squared image and
 *                       C_r(j) the Self-Convolution of Eq. eq:selfConv,
 *                       each evaluated on its own.
 * For integer input the two must agree bit for bit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BMO_OK 0
#define BMO_EINVAL -1
#define BMO_ENOMEM -3

#define BMO_SENTINEL_I64 ((int64_t)INT32_MAX)

typedef struct {
    int64_t di;   /* integer distance (uint8 input)  */
    double df;    /* double distance (float32 input) */
    int64_t off;  /* row-major offset y*W + x of the candidate top-left */
} bmo_cand;

static int cmp_int(const void* a, const void* b) {
    const bmo_cand* x = (const bmo_cand*)a;
    const bmo_cand* y = (const bmo_cand*)b;
    if (x->di != y->di) return x->di < y->di ? -1 : 1;
    if (x->off != y->off) return x->off < y->off ? -1 : 1;
    return 0;
}

static int cmp_dbl(const void* a, const void* b) {
    const bmo_cand* x = (const bmo_cand*)a;
    const bmo_cand* y = (const bmo_cand*)b;
    if (x->df != y->df) return x->df < y->df ? -1 : 1;
    if (x->off != y->off) return x->off < y->off ? -1 : 1;
    return 0;
}

/* Reference grid size per axis: floor((L - p) / s) + 1. */
int bmo_num_refs(int H, int W, int p, int s, int* n_ry, int* n_rx) {
    if (H < 1 || W < 1 || p < 1 || s < 1 || p > H || p > W) return BMO_EINVAL;
    if (n_ry) *n_ry = (H - p) / s + 1;
    if (n_rx) *n_rx = (W - p) / s + 1;
    return BMO_OK;
}

static int check_args(int H, int W, int C, int p, int win, int s, int K) {
    if (H < 1 || W < 1 || C < 1 || p < 1 || p > H || p > W) return 0;
    if (win < 1 || (win % 2) == 0 || s < 1 || K < 1) return 0;
    return 1;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Per reference: enumerate the clipped window, fill cand[], return count. */
static int window_bounds(int ry, int rx, int H, int W, int p, int h,
                         int* y0, int* y1, int* x0, int* x1) {
    *y0 = clampi(ry - h, 0, H - p);
    *y1 = clampi(ry + h, 0, H - p);
    *x0 = clampi(rx - h, 0, W - p);
    *x1 = clampi(rx + h, 0, W - p);
    return (*y1 - *y0 + 1) * (*x1 - *x0 + 1);
}

/* Emit the first min(K, n) sorted candidates, pad the rest. */
static void emit(const bmo_cand* c, int n, int K, int is_int,
                 int32_t* idx, int64_t* di, double* df) {
    for (int k = 0; k < K; ++k) {
        if (k < n) {
            idx[k] = (int32_t)c[k].off;
            if (is_int) di[k] = c[k].di; else df[k] = c[k].df;
        } else {
            idx[k] = -1;
            if (is_int) di[k] = BMO_SENTINEL_I64; else df[k] = INFINITY;
        }
    }
}

/*
 * Direct evaluation of Eq. equ:bm for one reference: explicit
 * sum over channels and patch pixels of the squared difference.
 */
static int match_one(const void* img, int is_int, int H, int W, int C, int p,
                     int h, int ry, int rx, bmo_cand* cand) {
    int y0, y1, x0, x1;
    window_bounds(ry, rx, H, W, p, h, &y0, &y1, &x0, &x1);
    int n = 0;
    for (int y = y0; y <= y1; ++y) {
        for (int x = x0; x <= x1; ++x) {
            int64_t si = 0;
            double sf = 0.0;
            for (int u = 0; u < p; ++u) {
                for (int v = 0; v < p; ++v) {
                    for (int c = 0; c < C; ++c) {
                        size_t ir = ((size_t)(ry + u) * W + (rx + v)) * C + c;
                        size_t ij = ((size_t)(y + u) * W + (x + v)) * C + c;
                        if (is_int) {
                            int64_t a = ((const uint8_t*)img)[ir];
                            int64_t b = ((const uint8_t*)img)[ij];
                            si += (a - b) * (a - b);
                        } else {
                            double a = ((const float*)img)[ir];
                            double b = ((const float*)img)[ij];
                            sf += (a - b) * (a - b);
                        }
                    }
                }
            }
            cand[n].di = si;
            cand[n].df = sf;
            cand[n].off = (int64_t)y * W + x;
            ++n;
        }
    }
    return n;
}

/*
 * Lemma 2 evaluation for one reference, each term computed on its own:
 *   ||X_j||^2  -- box sum of the squared image over the p x p x C patch,
 *   ||X_r||^2  -- the same box sum at the reference,
 *   C_r(j)     -- Eq. eq:selfConv: sum_l sum_m X_r(l, m) X(q+l-1, r+m-1),
 *                 summed over channels (S(.) of Eq. equ:self-convMM).
 */
static int selfconv_one(const void* img, int is_int, int H, int W, int C, int p,
                        int h, int ry, int rx, bmo_cand* cand) {
    int y0, y1, x0, x1;
    window_bounds(ry, rx, H, W, p, h, &y0, &y1, &x0, &x1);
    /* ||X_r||^2 */
    int64_t nri = 0;
    double nrf = 0.0;
    for (int u = 0; u < p; ++u)
        for (int v = 0; v < p; ++v)
            for (int c = 0; c < C; ++c) {
                size_t ir = ((size_t)(ry + u) * W + (rx + v)) * C + c;
                if (is_int) { int64_t a = ((const uint8_t*)img)[ir]; nri += a * a; }
                else { double a = ((const float*)img)[ir]; nrf += a * a; }
            }
    int n = 0;
    for (int y = y0; y <= y1; ++y) {
        for (int x = x0; x <= x1; ++x) {
            int64_t nji = 0, cri = 0;
            double njf = 0.0, crf = 0.0;
            /* h_X(j)^2: box sum of X^2 */
            for (int u = 0; u < p; ++u)
                for (int v = 0; v < p; ++v)
                    for (int c = 0; c < C; ++c) {
                        size_t ij = ((size_t)(y + u) * W + (x + v)) * C + c;
                        if (is_int) { int64_t b = ((const uint8_t*)img)[ij]; nji += b * b; }
                        else { double b = ((const float*)img)[ij]; njf += b * b; }
                    }
            /* C_r(j): correlation of the image with the reference patch */
            for (int l = 0; l < p; ++l)
                for (int m = 0; m < p; ++m)
                    for (int c = 0; c < C; ++c) {
                        size_t ir = ((size_t)(ry + l) * W + (rx + m)) * C + c;
                        size_t ij = ((size_t)(y + l) * W + (x + m)) * C + c;
                        if (is_int) {
                            cri += (int64_t)((const uint8_t*)img)[ir] *
                                   (int64_t)((const uint8_t*)img)[ij];
                        } else {
                            crf += (double)((const float*)img)[ir] *
                                   (double)((const float*)img)[ij];
                        }
                    }
            cand[n].di = nji + nri - 2 * cri;
            cand[n].df = njf + nrf - 2.0 * crf;
            cand[n].off = (int64_t)y * W + x;
            ++n;
        }
    }
    return n;
}

/*
 * Shared driver.  `refs` lists the row-major reference indices to compute
 * (NULL = all n_ry * n_rx of them); output row i belongs to refs[i].
 */
static int run(const void* img, int is_int, int use_selfconv, int H, int W, int C,
               int p, int win, int s, int K, const int32_t* refs, int n_refs,
               int32_t* out_idx, int64_t* out_di, double* out_df, int nthreads) {
    if (!img || !out_idx || (is_int ? !out_di : !out_df)) return BMO_EINVAL;
    if (!check_args(H, W, C, p, win, s, K)) return BMO_EINVAL;
    int n_ry, n_rx;
    bmo_num_refs(H, W, p, s, &n_ry, &n_rx);
    int total = n_ry * n_rx;
    int n = refs ? n_refs : total;
    if (refs) {
        for (int i = 0; i < n; ++i)
            if (refs[i] < 0 || refs[i] >= total) return BMO_EINVAL;
    }
    int h = (win - 1) / 2;
    int err = BMO_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        bmo_cand* cand = (bmo_cand*)malloc(sizeof(bmo_cand) * (size_t)win * (size_t)win);
        if (!cand) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = BMO_ENOMEM;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int i = 0; i < n; ++i) {
                int r = refs ? refs[i] : i;
                int ry = (r / n_rx) * s, rx = (r % n_rx) * s;
                int m = use_selfconv
                            ? selfconv_one(img, is_int, H, W, C, p, h, ry, rx, cand)
                            : match_one(img, is_int, H, W, C, p, h, ry, rx, cand);
                qsort(cand, (size_t)m, sizeof(bmo_cand), is_int ? cmp_int : cmp_dbl);
                emit(cand, m, K, is_int, out_idx + (size_t)i * K,
                     is_int ? out_di + (size_t)i * K : NULL,
                     is_int ? NULL : out_df + (size_t)i * K);
            }
            free(cand);
        }
    }
    return err;
}

int bmo_match_u8(const uint8_t* img, int H, int W, int C, int p, int win, int s,
                 int K, const int32_t* refs, int n_refs, int32_t* out_idx,
                 int64_t* out_dist, int nthreads) {
    return run(img, 1, 0, H, W, C, p, win, s, K, refs, n_refs, out_idx, out_dist,
               NULL, nthreads);
}

int bmo_match_f32(const float* img, int H, int W, int C, int p, int win, int s,
                  int K, const int32_t* refs, int n_refs, int32_t* out_idx,
                  double* out_dist, int nthreads) {
    return run(img, 0, 0, H, W, C, p, win, s, K, refs, n_refs, out_idx, NULL,
               out_dist, nthreads);
}

int bmo_selfconv_u8(const uint8_t* img, int H, int W, int C, int p, int win, int s,
                    int K, const int32_t* refs, int n_refs, int32_t* out_idx,
                    int64_t* out_dist, int nthreads) {
    return run(img, 1, 1, H, W, C, p, win, s, K, refs, n_refs, out_idx, out_dist,
               NULL, nthreads);
}

int bmo_selfconv_f32(const float* img, int H, int W, int C, int p, int win, int s,
                     int K, const int32_t* refs, int n_refs, int32_t* out_idx,
                     double* out_dist, int nthreads) {
    return run(img, 0, 1, H, W, C, p, win, s, K, refs, n_refs, out_idx, NULL,
               out_dist, nthreads);
}

/*
 * Distance of one explicit (reference, candidate) pair by the definition
 * (Eq. equ:bmMetric_app), for sampled parity checks at full size.
 * ry, rx, cy, cx are top-left corners.  Returns the distance through *d.
 */
int bmo_pair_u8(const uint8_t* img, int H, int W, int C, int p, int ry, int rx,
                int cy, int cx, int64_t* d) {
    if (!img || !d || ry < 0 || rx < 0 || cy < 0 || cx < 0 || ry + p > H ||
        cy + p > H || rx + p > W || cx + p > W)
        return BMO_EINVAL;
    int64_t sum = 0;
    for (int u = 0; u < p; ++u)
        for (int v = 0; v < p; ++v)
            for (int c = 0; c < C; ++c) {
                int64_t a = img[((size_t)(ry + u) * W + (rx + v)) * C + c];
                int64_t b = img[((size_t)(cy + u) * W + (cx + v)) * C + c];
                sum += (a - b) * (a - b);
            }
    *d = sum;
    return BMO_OK;
}

int bmo_pair_f32(const float* img, int H, int W, int C, int p, int ry, int rx,
                 int cy, int cx, double* d) {
    if (!img || !d || ry < 0 || rx < 0 || cy < 0 || cx < 0 || ry + p > H ||
        cy + p > H || rx + p > W || cx + p > W)
        return BMO_EINVAL;
    double sum = 0.0;
    for (int u = 0; u < p; ++u)
        for (int v = 0; v < p; ++v)
            for (int c = 0; c < C; ++c) {
                double a = img[((size_t)(ry + u) * W + (rx + v)) * C + c];
                double b = img[((size_t)(cy + u) * W + (cx + v)) * C + c];
                sum += (a - b) * (a - b);
            }
    *d = sum;
    return BMO_OK;
}

int bmo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
