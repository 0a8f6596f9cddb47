/*
 * bm.h -- C ABI of the GB300 (sm_103a) Self-Convolution block matcher.
 *
 * The operation (arXiv 2006.13714, "Exploiting Non-Local Priors via
 * Self-Convolution"):
 *
 *   For every reference patch X_r and every candidate patch X_j whose
 *   top-left corner lies in the search window of X_r, the squared distance
 *     d(r, j) = ||X_j - X_r||_F^2                           (§III-A, Eq. equ:bm)
 *             = ||X_j||^2 + ||X_r||^2 - 2 <X_r, X_j>        (§III-B, Lemma 2)
 *   where <X_r, X_j> is the Self-Convolution C_r(j) of Eq. eq:selfConv
 *   (restricted to the window as in the footnote to Eq. eq:unifySelfConv)
 *   and ||X_j||^2 is a box filter of the squared image (the h_X (.) h_X
 *   vector of §III-B).  Multi-channel patches sum the distance over
 *   channels (§IV, S(.) in Eq. equ:self-convMM).  The output per reference
 *   is the K candidates of smallest distance (Theorem 1: the l0 projection
 *   of b = vec(C_r) - 0.5 h_X (.) h_X keeps the K largest entries).
 *
 * Geometry (readings of the paper, identical in the oracle):
 *   - image: H x W x C, channels innermost, row-major, contiguous;
 *   - candidate top-left grid G = [0, H-p] x [0, W-p];
 *   - reference grid R = {(s*a, s*b)} in G, row-major;
 *     n_ry = floor((H-p)/s) + 1, n_rx = floor((W-p)/s) + 1;
 *   - window: top-left offsets dy, dx in [-h, h], h = (window-1)/2,
 *     window odd, clipped to G (no padding, no shifting);
 *   - order: distance ascending, then row-major offset y*W + x ascending;
 *   - if the clipped window holds fewer than K candidates the tail of the
 *     row is idx = -1, dist = INT32_MAX (uint8) / +inf (float32).
 *
 * Outputs: out_idx int32 [n_ry*n_rx][K] holds the candidate top-left as the
 * row-major pixel offset y*W + x; out_dist is int32 (uint8 input, exact) or
 * float32 (float32 input) of the same shape.
 *
 * Precision: uint8 distances are exact integers and the indices are
 * bit-identical to the brute-force definition.  float32 distances are
 * within 1e-4 relative of the exact (double) value; the K-set equals the
 * exact one except for swaps among candidates whose exact distances differ
 * by less than that tolerance.  Non-finite float32 pixels are not checked.
 *
 * Memory: every pointer named img / out_* in a device entry point is a
 * device pointer owned by the caller; the library never frees it.  The
 * library allocates its own workspace (inside the context's budget).
 *
 * Errors: every entry point returns a bm_status; nothing throws across the
 * ABI.  On BM_ERR_INVALID / BM_ERR_UNSUPPORTED no kernel is launched and no
 * output is written.  bm_last_error() returns the calling thread's last
 * message for that context.
 */
#ifndef BM_H_
#define BM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bm_ctx bm_ctx;
/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* bm_stream;

typedef enum { BM_U8 = 0, BM_F32 = 1 } bm_dtype;

typedef enum {
    BM_OK = 0,
    BM_ERR_INVALID = -1,     /* bad argument; nothing launched            */
    BM_ERR_UNSUPPORTED = -2, /* valid but not implemented (e.g. p*p*C>256)*/
    BM_ERR_OOM = -3,         /* workspace exceeds the context budget      */
    BM_ERR_CUDA = -4,        /* a CUDA call failed; see bm_last_error     */
    BM_ERR_TIMEOUT = -5,     /* a bounded device wait ran out             */
    BM_ERR_BUSY = -6,        /* request alone exceeds the budget          */
    BM_ERR_NOT_FOUND = -7,   /* unknown ticket                            */
    BM_ERR_TOO_LARGE = -8    /* job exceeds bm_match_static's scratch     */
} bm_status;

/* Algorithm selector for bm_set_algo. */
typedef enum {
    BM_ALGO_AUTO = 0,        /* tensor-core Self-Convolution when supported */
    BM_ALGO_SELFCONV_TC = 1, /* tcgen05 cross term + box filter + top-K     */
    BM_ALGO_DIRECT = 2       /* plain FP32 CUDA-core sum of (X_r - X_j)^2   */
} bm_algo;

/* One block-matching job; same fields as bm_match. */
typedef struct {
    const void* img;
    int H, W, C;
    bm_dtype dtype;
    int patch, window, stride, K;
    int32_t* out_idx;
    void* out_dist;
} bm_request;

/* Counters accumulated over the context's life (host-read, best effort). */
typedef struct {
    uint64_t matches;         /* images matched                                  */
    uint64_t refs;            /* reference patches matched                       */
    uint64_t rerank_overflow; /* float32 refs whose boundary band left the pool  */
    uint64_t fp64_rechecks;   /* float32 boundary ties re-ranked in FP64         */
    uint64_t bound_violations;/* float32 pool entries outside the stated error bound (expected 0) */
    uint64_t tc_jobs;         /* images matched on the tensor-core path          */
} bm_stats;

/*
 * Create a context on CUDA device `device`.  mem_budget_bytes bounds the
 * library's own device workspace (0 = 40 GiB).  tune_cache (nullable) is
 * a file path where tuned tile choices are read from and written to: with
 * it, the first job of each class (dtype, channels, patch, window, stride,
 * K) times every tile configuration of the tensor-core kernel on its own
 * data and keeps the fastest whose output equals the default's.
 * Returns BM_OK and *out, or an error (then *out is NULL).
 */
int bm_create(bm_ctx** out, int device, size_t mem_budget_bytes, const char* tune_cache);

/* Destroy a context: drains its serving queue, frees its workspace. NULL is a no-op. */
void bm_destroy(bm_ctx* ctx);

/* Last error message of the calling thread for ctx ("" if none). Never NULL. */
const char* bm_last_error(bm_ctx* ctx);

/* Reference grid size, host only: n_ry = floor((H-p)/s)+1, n_rx likewise. */
int bm_num_refs(int H, int W, int patch, int stride, int* n_ry, int* n_rx);

/*
 * K-nearest block matching of one image, asynchronous on `stream`
 * (device pointers; see the file header for layout and conventions).
 * Validation: 1 <= patch <= min(H, W); window odd, 1 <= window <= 127;
 * stride >= 1; 1 <= K <= 128; 1 <= C <= 8; non-null pointers (else
 * BM_ERR_INVALID); patch*patch*C <= 256 and H*W < 2^31 (else
 * BM_ERR_UNSUPPORTED).
 */
int bm_match(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype,
             int patch, int window, int stride, int K,
             int32_t* out_idx, void* out_dist, bm_stream stream);

/*
 * Same result through the plain FP32 CUDA-core direct-distance kernel
 * (explicit sum of squared differences, Eq. equ:bmMetric_app): the
 * comparison baseline.  Same arguments and conventions as bm_match.
 */
int bm_match_direct(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype,
                    int patch, int window, int stride, int K,
                    int32_t* out_idx, void* out_dist, bm_stream stream);

/*
 * Host-buffer variant: img, out_idx and out_dist are HOST pointers.  The
 * call copies the image to the device, matches, copies the results back
 * and returns after they have landed (synchronous).
 */
int bm_match_host(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype,
                  int patch, int window, int stride, int K,
                  int32_t* out_idx, void* out_dist);

/*
 * Host-buffer batch: n jobs whose img / out_idx / out_dist are HOST pointers
 * (same fields and conventions as bm_match_batch otherwise).  Consecutive
 * jobs are grouped in chunks (up to 16 jobs or 96 MB of staging) that run in
 * two pipelines of (host-to-device copy, batched match, device-to-host copy)
 * on the context's own streams, so the copies of one chunk overlap the
 * matching of the next; the staging buffers are cached in the context.
 * Returns after every result has landed (synchronous), with the check of
 * bm_check.  Copies overlap only for page-locked host buffers.
 */
int bm_match_host_batch(bm_ctx* ctx, const bm_request* reqs, int n);

/*
 * Match n independent jobs (any mix of sizes, channel counts, dtypes and
 * parameters) with one persistent launch per kernel stage, asynchronous on
 * `stream`.  Same per-job conventions as bm_match.  On a stream other than
 * the legacy default stream, and with stage timing off, a call with the same
 * job list (same descriptors) as the previous call on that stream replays a
 * captured CUDA graph of the whole batch.
 */
int bm_match_batch(bm_ctx* ctx, const bm_request* reqs, int n, bm_stream stream);

/*
 * Failure detection.  Every wait inside the tensor-core kernel is bounded
 * (2 s); when one runs out, that CTA stops, waits for its copies and MMAs in
 * flight, frees its tensor memory, and records the wait site in the
 * context's sticky fault word (the outputs of that job are then invalid).
 * bm_check synchronises `stream` and reports that word: BM_OK, or
 * BM_ERR_TIMEOUT with the site in bm_last_error (the word is cleared, the
 * context stays usable).  bm_match_host performs the same check before it
 * returns.  Asynchronous entry points cannot report it themselves; call
 * bm_check after the work of interest.
 */
int bm_check(bm_ctx* ctx, bm_stream stream);

/*
 * Test hook for the above: mode 1 makes the next tensor-core launch of
 * bm_match (not bm_match_batch) withhold one stage publication in one CTA,
 * so that a bounded wait runs out; mode 0 disarms it.  One-shot.
 */
int bm_set_fault_injection(bm_ctx* ctx, int mode);

/* Select the algorithm used by bm_match / bm_match_batch / bm_submit. */
int bm_set_algo(bm_ctx* ctx, bm_algo algo);

/*
 * Serving: enqueue a request (the descriptor is copied, the buffers are
 * not: they must stay alive until bm_poll reports done).  Requests are
 * admitted under the memory budget as earlier ones finish and run
 * concurrently on the context's streams.  BM_ERR_BUSY: the request alone
 * exceeds the budget.  *ticket identifies it for bm_poll.
 */
int bm_submit(bm_ctx* ctx, const bm_request* req, uint64_t* ticket);

/*
 * Non-blocking completion check (never waits for the serving thread's
 * launches).  *done = 1 once the request finished; *status then holds its
 * bm_status: BM_OK, BM_ERR_TIMEOUT when a bounded device wait of its
 * tensor-core kernel ran out (its outputs are incomplete; the wait site is
 * in bm_last_error of the polling thread), BM_ERR_OOM or BM_ERR_CUDA.  A
 * ticket is released by the first poll that reports done.  Unknown ticket:
 * BM_ERR_NOT_FOUND.
 */
int bm_poll(bm_ctx* ctx, uint64_t ticket, int* done, int* status);

/* Read the context counters. */
int bm_get_stats(bm_ctx* ctx, bm_stats* out);

/* Kernel stages timed by bm_set_timing. */
enum {
    BM_STAGE_PLANES = 0, /* bf16 operand planes                          */
    BM_STAGE_BOX = 1,    /* (a1) box filter of the squared image         */
    BM_STAGE_TC = 2,     /* (a3-a5) tensor-core cross term + top-K       */
    BM_STAGE_RERANK = 3, /* (a6) float32 boundary re-rank                */
    BM_STAGE_DIRECT = 4, /* plain FP32 direct-distance kernel            */
    BM_NUM_STAGES = 5
};

typedef struct {
    uint64_t launches[BM_NUM_STAGES]; /* kernel launches timed per stage */
    double ms[BM_NUM_STAGES];         /* summed device time per stage    */
} bm_timing;

/*
 * Stage timing: while enabled, every kernel launch of the context is
 * bracketed by CUDA events on its own stream.  bm_get_timing waits for the
 * recorded events, adds their elapsed times into *out (accumulated since
 * the last reset) and, if reset != 0, clears the totals.
 */
int bm_set_timing(bm_ctx* ctx, int enable);
int bm_get_timing(bm_ctx* ctx, bm_timing* out, int reset);

/*
 * Patch groups (§IV, the group matrix after Eq. equ:self-convMM):
 * Y_r = [y_S(1), ..., y_S(K)], the K matched patches of reference r, as
 *   out_groups[r][k][(u*patch + v)*C + c] = img[y + u][x + v][c]
 * where idx[r][k] = y*W + x (the layout bm_match writes: r = ry*n_rx + rx
 * over the n_ry x n_rx reference grid).  An index that is not a top-left
 * of the candidate grid (-1, or out of range) gives a zero patch.
 * img: device, H x W x C, uint8 or float32 (dtype); idx: device int32
 * [n_ry*n_rx][K]; out_groups: device, same element type as img,
 * [n_ry*n_rx][K][patch*patch*C], caller-owned.  Asynchronous on `stream`.
 * Validation: 1 <= C <= 8, 1 <= patch <= min(H, W), n_ry, n_rx >= 0,
 * 1 <= K <= 128, non-null pointers (BM_ERR_INVALID, nothing launched);
 * H*W < 2^31 and patch*patch*C <= 256 (BM_ERR_UNSUPPORTED).  An empty
 * grid launches nothing.
 */
int bm_gather_groups(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype,
                     int patch, const int32_t* idx, int n_ry, int n_rx, int K,
                     void* out_groups, bm_stream stream);

/*
 * Image reconstruction (§IV, "Image Reconstruction"): every patch
 * groups[r][k] (layout of bm_gather_groups, float32) is deposited back at
 * idx[r][k] and every pixel is divided by the number of deposited patches
 * that contain it; with weights (nullable, float32 [n_ry*n_rx][K]) by their
 * sum instead:
 *   out_img[y][x][c] = sum w * Z / sum w,   out_weight[y][x] = sum w,
 * both over the patches covering (y, x); 0 where no patch covers the pixel
 * (or the weights sum to 0).  Patches whose index is not a top-left of the
 * candidate grid are skipped.  out_img (H x W x C) and out_weight (H x W)
 * are device float32 buffers owned by the caller; both are overwritten.
 * The sums are accumulated in float32 in an unspecified order (atomics):
 * each pixel is within (n + 1) * 2^-23 * sum |w Z| / |sum w| of the exact
 * value, n the number of covering patches; unweighted counts are exact.
 * Same validation as bm_gather_groups (out_img and out_weight required).
 */
int bm_aggregate(bm_ctx* ctx, const float* groups, const int32_t* idx, const float* weights,
                 int n_ry, int n_rx, int K, int H, int W, int C, int patch,
                 float* out_img, float* out_weight, bm_stream stream);

/*
 * 3-D block matching across channels (§IV: the 3-D Self-Convolution on
 * patches of depth d < C, searched across channels, the channel sum S(.)
 * omitted).  A 3-D patch at (y, x, c) holds X[y + u][x + v][c + t] for
 * u, v < patch, t < depth.  References: the spatial grid of bm_match at every
 * channel offset c_r in [0, C - depth]; row index
 * (ry * n_rx + rx) * (C - depth + 1) + c_r.  Candidates: the clipped spatial
 * window of bm_match at every channel offset.  out_idx int32
 * [n_ry*n_rx*(C-depth+1)][K]: offsets (y * W + x) * C + c (the flat HWC index
 * of the candidate's first element), nearest first by (distance, offset),
 * -1 padding; out_dist int32 (uint8, exact; INT32_MAX padding) or float32
 * (float32 sums of squared differences; +inf padding).  Device pointers,
 * asynchronous on `stream`.  Validation as bm_match plus 1 <= depth <= C
 * (BM_ERR_INVALID); patch*patch*depth <= 128, K <= 32, H*W*C < 2^31 and a
 * search region that fits in shared memory (BM_ERR_UNSUPPORTED).
 */
int bm_match_3d(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                int depth, int window, int stride, int K, int32_t* out_idx, void* out_dist,
                bm_stream stream);

/*
 * Block matching by normalized cross-correlation (§III-A, Eq. equ:cor;
 * Lemma 1 and Theorem 1, case 3): over the same clipped search windows and
 * reference grid as bm_match, the K candidates with the largest
 *   ncc(r, j) = <X_r, X_j> / (||X_r||_F ||X_j||_F)
 * (the uncentred cosine; a patch of zero norm scores 0), ties broken by the
 * smaller row-major offset.  out_idx int32 [n_ry*n_rx][K] (offsets y*W + x,
 * best first, -1 padding), out_score float32 (-inf padding).  uint8: the
 * ranking is exact (integer cross terms and norms compared in 128-bit
 * integers) and the scores are the correctly rounded quotient of exact
 * integers; float32: ranked by the float32 score, within 2e-5 of the exact
 * cosine.  Device pointers, asynchronous on `stream`.  Validation as
 * bm_match (BM_ERR_INVALID / BM_ERR_UNSUPPORTED); additionally K <= 64 and a
 * search region that fits in shared memory (BM_ERR_UNSUPPORTED).
 */
int bm_match_ncc(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                 int window, int stride, int K, int32_t* out_idx, float* out_score,
                 bm_stream stream);

/*
 * Non-local means (§III-A, Eq. equ:nlm; Prop. 1 gives the same weights
 * through Self-Convolution), over the same clipped search windows and
 * reference grid as bm_match.  For every reference r (row-major over the
 * n_ry x n_rx grid) and every candidate j of its window:
 *   w_r(j) = exp(-||X_j - X_r||_F^2 / b^2),  Theta_r = sum_j w_r(j),
 *   out_est[r][(u*patch + v)*C + c] = sum_j w_r(j) X_j[u][v][c] / Theta_r,
 *   out_theta[r] = Theta_r   (nullable; >= 1, the reference is a candidate).
 * img: device, H x W x C, uint8 or float32; out_est / out_theta: device
 * float32, caller-owned.  Computed in float32 (distances directly, packed
 * FP32); each estimate is within about 2^-17 of the data range of the
 * exact value.  Asynchronous on `stream`.
 * Validation: geometry as bm_match, b > 0 and finite, non-null img and
 * out_est (BM_ERR_INVALID, nothing launched); patch*patch*C <= 64 and a
 * search region that fits in shared memory (BM_ERR_UNSUPPORTED).
 */
int bm_nlm(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
           int window, int stride, float b, float* out_est, float* out_theta, bm_stream stream);

/*
 * bm_match_static -- bm_match without any allocation.
 *
 * The paper has no counterpart: this entry point serves callers that must
 * not allocate device memory while they run.  cudaMalloc and cudaFree
 * synchronise the whole device, which stalls a latency-bound loop, and in a
 * process whose device memory is already held by another allocator (a
 * framework's caching allocator, a fixed arena) a fresh allocation can fail
 * part-way through a run.  bm_match_static needs no context and calls no
 * cudaMalloc, cudaFree or other allocating routine: every intermediate
 * buffer (bf16 operand planes, patch norms, float32 candidate pool, the
 * column-part lists of the classes that need them, status word, counters)
 * is carved from one array in device memory of
 * BM_STATIC_SCRATCH_BYTES (16 MiB).  The array belongs to a module of the
 * library that CUDA loads lazily (its default): the first symbol lookup on a
 * device reserves it -- bm_static_init(), or else the first bm_match_static
 * call there -- and that first step can fail when device memory is already
 * full.  Call bm_static_init() at start-up (or run with
 * CUDA_MODULE_LOADING=EAGER) to reserve it before memory fills up.
 *
 * Same arguments, conventions, validation and results as bm_match with the
 * default algorithm (device pointers; asynchronous on `stream`).  A job
 * whose working set (bm_static_scratch_bytes) exceeds the array returns
 * BM_ERR_TOO_LARGE with nothing launched; bm_last_error(NULL) says how many
 * bytes it needed.  For reference, a 512 x 512 float32 image with patch 8,
 * stride 3, window 39, K 16 needs about 11.7 MB.
 *
 * Set-up: the first call on a device (the current device) looks up the
 * array's address there with cudaGetSymbolAddress.  Make that first call
 * before any stream capture begins.
 *
 * Sharing: every call on a device uses the same array.  Each call first
 * clears the part that must start at zero (status word and counters) on
 * `stream`; everything else is overwritten before it is read.  Calls whose
 * work overlaps on the GPU (different streams with no ordering between
 * them, or calls from several threads) race on the array and give wrong
 * results: order them on one stream, or with events.
 */
#define BM_STATIC_SCRATCH_BYTES ((size_t)16 << 20)

/* Reserves the static array (and the fault word below) on the current
 * device and looks up their addresses; later calls there do nothing.
 * Returns BM_OK or BM_ERR_CUDA (module load or lookup failed, e.g. device
 * memory is full).  Host only; no stream work. */
int bm_static_init(void);

/* Timeout report of bm_match_static on the current device.  A bounded
 * device wait of the tensor-core kernel (2 s per wait) that runs out leaves
 * that call's outputs incomplete; the kernel records the wait site in a
 * sticky per-device word, which the calls never clear.  bm_static_check
 * synchronises `stream`, reads the word into a host int and clears it:
 * BM_OK (no timeout since the last check) or BM_ERR_TIMEOUT with the site in
 * bm_last_error(NULL).  It allocates nothing.  Check after the calls whose
 * results you use, on the stream they ran on. */
int bm_static_check(bm_stream stream);

/* Test hook: mode 1 makes the next bm_match_static call's tensor-core kernel
 * withhold its first stage once, so that a bounded wait runs out and the
 * timeout path above is taken (no GPU fault: the kernel returns normally).
 * 0 cancels.  BM_ERR_INVALID for any other mode. */
int bm_static_set_fault_injection(int mode);

/*
 * Device workspace (bytes) a context allocates for this job with the
 * default algorithm: operand planes, norms, float32 candidate pool, window-
 * split part lists, status words.  0 when the job runs on the direct kernel
 * (no workspace) or the arguments are invalid.  Admission under a context's
 * memory budget (bm_create, bm_submit) counts these bytes.  Host only.
 */
size_t bm_workspace_bytes(int H, int W, int C, bm_dtype dtype, int patch, int window, int stride,
                          int K);

/*
 * Window split (host only, no device work): the number of parts each tile's
 * search window is split into when this job runs alone through bm_match,
 * bm_match_batch or bm_submit on the tensor-core path.  A launch whose
 * tiles (128 references each) are fewer than the GPU's 152 SMs
 * splits each tile's union of windows into 2 or 4 column ranges that
 * separate CTAs run; each part keeps its own top-K list (float32: pool),
 * and a merge kernel combines them, so results are identical to an unsplit
 * run.  A launch with enough tiles (a batch of many images) does not split.
 * Classes whose staged tile does not fit shared memory whole (float32 four-
 * channel at window 61 with K above 16 or patch 7; large windows) always
 * run split into 2, 3 or 4 contiguous column parts, each staging only its
 * own columns, in every entry point, bm_match_static included.  Returns 1
 * (no split), 2, 3 or 4; 0 for invalid arguments.  Apart from those
 * classes, bm_match_static never splits.
 */
int bm_window_split(int H, int W, int C, bm_dtype dtype, int patch, int window, int stride, int K);

/* Scratch bytes bm_match_static needs for this job (0 if the arguments are
 * invalid or unsupported).  Host only. */
size_t bm_static_scratch_bytes(int H, int W, int C, bm_dtype dtype,
                               int patch, int window, int stride, int K);

int bm_match_static(const void* img, int H, int W, int C, bm_dtype dtype,
                    int patch, int window, int stride, int K,
                    int32_t* out_idx, void* out_dist, bm_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* BM_H_ */
