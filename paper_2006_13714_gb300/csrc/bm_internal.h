// bm_internal.h -- shared declarations of the CUDA block-matching library.
//
// Geometry of one job (readings shared with the public header bm.h):
//   image H x W x C (HWC, row-major); patch p; stride s; window 2h+1;
//   candidate top-left grid G = [0, H-p] x [0, W-p];
//   reference grid R = {(s*a, s*b)} in G; n_ry = (H-p)/s + 1, n_rx = (W-p)/s + 1.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

struct bm_ctx;

namespace bm {

// n / d for every n in [0, 2^31) by a multiply-high and two shifts (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994;
// the round-up method): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) with t = mulhi(m, n).
struct FastDiv {
    unsigned m;
    int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.m = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s1 = l > 0 ? 1 : 0;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}

__device__ __forceinline__ int fast_div(int n, const FastDiv& f) {
    const unsigned t = __umulhi((unsigned)n, f.m);
    return (int)((t + (((unsigned)n - t) >> f.s1)) >> f.s2);
}

// A warp's top-K list of 64-bit keys, smaller is better: lane i holds entry
// i in rank order (lanes >= K hold nothing of use) and `kth` is entry K - 1
// on every lane (all ones while the list is not full).  offer() screens the
// 32 lanes' keys with one ballot against the K-th and inserts each one that
// still beats it at its rank (a ballot count) with one shuffle of the list.
// Every lane of the warp must call it.
__device__ __forceinline__ void warp_list_offer(unsigned long long key, unsigned long long& mine,
                                                unsigned long long& kth, int lane, int K) {
    unsigned mask = __ballot_sync(0xffffffffu, key < kth);
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const unsigned long long b = __shfl_sync(0xffffffffu, key, src);
        if (!(b < kth)) continue;  // the K-th moved past it
        const int pos = __popc(__ballot_sync(0xffffffffu, lane < K && mine < b));
        const unsigned long long up = __shfl_up_sync(0xffffffffu, mine, 1);
        if (lane == pos) mine = b;
        else if (lane > pos) mine = up;
        kth = __shfl_sync(0xffffffffu, mine, K - 1);
    }
}

// Device ordinal of a context (bm_api.cu).
int ctx_device(const ::bm_ctx* ctx);
// For entry points in other files (bm_api.cu): the per-stream workspace of
// at least `bytes` (budget-checked, stream-ordered), the sticky timeout
// word, the device counters ([0] overflow, [1] fp64 rechecks, [2] bound
// violations), the tensor-core job counter, and whether the context's
// algorithm allows the tensor-core path.
int ctx_workspace(::bm_ctx* ctx, cudaStream_t st, size_t bytes, void** out);
int* ctx_fault_word(::bm_ctx* ctx);
unsigned long long* ctx_counters(::bm_ctx* ctx);
void ctx_count_tc_job(::bm_ctx* ctx);
bool ctx_uses_tc(::bm_ctx* ctx);

constexpr int kMaxK = 128;        // largest K served
constexpr int kMaxPatchElems = 256;  // p*p*C limit of every kernel
constexpr int kMaxWindow = 127;   // largest odd window
constexpr int kMaxC = 8;

enum DType : int { kU8 = 0, kF32 = 1 };

struct Geom {
    int H, W, C, dtype;
    int p, win, h, s, K;
    int n_ry, n_rx, nR;
    int Hc, Wc;          // candidate grid extent: H-p+1, W-p+1
    // bf16 operand planes (tensor-core path)
    int Cp;              // channels padded to 1, 2, 4 or 8
    int pw;              // 16-byte chunks per patch row, even unless 1
    int p_eff;           // patch rows fed to the MMA (p, rounded up to even if pw == 1)
    int plane_pitch;     // elements per plane row (multiple of 8)
    int plane_rows;      // rows per plane (H + padding)
    int L;               // float32 candidate pool per reference
    // normalized cross-correlation (bm_match_ncc on tensor cores): uncentred
    // operands, no norm K-step, scores a_j / ||X_j|| in the epilogue, a pool
    // of L for both dtypes (set by the NCC entry point after make_geom)
    int ncc = 0;
};

// Fill g from the arguments; returns 0 or a negative bm_status.
int make_geom(Geom& g, int H, int W, int C, int dtype, int p, int win, int s, int K);

// Workspace byte counts of one job (tensor-core path).
size_t plane_bytes(const Geom& g);       // one bf16 plane
size_t nrm_bytes(const Geom& g);         // candidate norms
size_t pool_bytes(const Geom& g);        // float32 candidate pool
size_t nsp_bytes(const Geom& g);         // split candidate norms (16 bytes each)

// ---- kernels (each launcher returns cudaGetLastError()) ----

// One image's preparation (centre, planes, box filter) inside a batch.
struct PrepJob {
    const void* img;
    float* center;            // centring offset (written by the centre kernel)
    int* status;              // nullable: device error word, zeroed by the centre kernel
    uint16_t* plane0;         // bf16 planes
    uint16_t* plane1;
    void* nrm;                // norms [Hc][Wc]
    uint16_t* nsp;            // nullable: split norms [Wc][Hc][8]
    int H, W, C, Cp, p, Hc, Wc, plane_pitch, plane_rows, dtype;
    // NCC: uncentred planes (uint8 too gets a zero lo plane), uncentred norms,
    // and nsp holding 1 / ||X_j|| (float, first 4 bytes of each 16) instead of
    // the split norm pieces
    int ncc = 0;
};
PrepJob make_prep_job(const Geom& g, const void* img, float* center, uint16_t* plane0,
                      uint16_t* plane1, void* nrm, uint16_t* nsp);
// Batched forms (one launch per stage for up to 64 jobs; the centre must
// precede the planes and the box filter).
cudaError_t launch_center_batch(const PrepJob* jobs, int n, cudaStream_t st);
cudaError_t launch_planes_batch(const PrepJob* jobs, int n, cudaStream_t st);
cudaError_t launch_box_batch(const PrepJob* jobs, int n, cudaStream_t st);

// Centring offset c of the operands (distances are shift-invariant):
// uint8 -> 128 (constant, nothing written but a zero), float32 -> a sampled
// image mean written to *center.
cudaError_t launch_center(const Geom& g, const void* img, float* center, cudaStream_t st);

// (a1) box filter of the squared centred image:
//      nrm[y][x] = sum_{u,v<p, c<C} (X[y+u][x+v][c] - c0)^2
//      int32 (uint8, exact) or float32 (float32, compensated summation).
// nsp (nullable): the same values split into bf16 pieces for the tensor-core
// norm K-step, column-major nsp[x][y][8]: uint8 (hi, mid, lo, 0...) exact,
// float32 (hi, mid, lo, hi, mid, lo, 0, 0).
cudaError_t launch_boxfilter(const Geom& g, const void* img, const float* center, void* nrm,
                             uint16_t* nsp, cudaStream_t st);

// bf16 operand planes of the centred image: uint8 -> one exact plane;
// float32 -> hi and lo planes with x - c0 ~= hi + lo (hi = RN_bf16, lo = RN_bf16(rest)).
cudaError_t launch_planes(const Geom& g, const void* img, const float* center, uint16_t* plane0,
                          uint16_t* plane1, cudaStream_t st);

// Plain FP32 CUDA-core direct-distance block matcher (comparison baseline).
cudaError_t launch_direct(const Geom& g, const void* img, int32_t* out_idx, void* out_dist,
                          cudaStream_t st);

// (a3-a5) tensor-core cross term + distance assembly + top-K.
// uint8: writes the final out_idx / out_dist.  float32: writes the candidate
// pool (pool_idx, pool_score) of L entries per reference.
struct TcArgs {
    const uint16_t* plane0;   // bf16 hi (or exact uint8) plane
    const uint16_t* plane1;   // bf16 lo plane (float32 only)
    const void* nrm;          // int32 or float32 norms [Hc][Wc]
    const uint16_t* nsp;      // split norms [Wc][Hc][8] bf16 (launch_boxfilter)
    int32_t* out_idx;         // uint8: final indices
    int32_t* out_dist;        // uint8: final distances
    int32_t* pool_idx;        // float32: candidate pool offsets [nR][L]
    float* pool_score;        // float32: candidate pool scores  [nR][L]
    int* status;              // device error word (0 = ok)
    int* fault = nullptr;     // nullable: context-wide sticky word, first timeout code kept
    int inject = 0;           // test hook: 1 = the producer skips publishing its first stage
    // window split (nullable): room for up to `wsplit` part lists of the job
    // ([wsplit][nR][N] offsets and distances / score bits, N = K for uint8,
    // L for float32).  A launch that leaves SMs idle splits each tile's
    // window into parts that separate CTAs run, then merges the parts' lists
    // into the outputs (uint8) or the pool (float32).
    int wsplit = 1;
    int32_t* split_idx = nullptr;
    int32_t* split_val = nullptr;
};
cudaError_t launch_tc(const Geom& g, const TcArgs& a, cudaStream_t st);
// Several jobs in persistent launches (consecutive jobs of one class share a
// launch, up to 64 jobs each); *nlaunch (nullable) = kernel launches made.
cudaError_t launch_tc_batch(const Geom* gs, const TcArgs* as, int n, cudaStream_t st,
                            int* nlaunch = nullptr, const int* choices = nullptr);
// Tile configurations the tensor-core kernel can run a job shape with
// (choices[i] in launch_tc_batch: 0 .. n-1; -1 = the built-in heuristic).
int tc_num_choices(const Geom& g);
bool tc_supported(const Geom& g);
// float32 pool scores of the tensor-core pass are rounded up by less than
// 2^bits ulp (0: exact float32 scores).
int tc_score_bits(const Geom& g);
bool tc_same_class(const Geom& a, const Geom& b);
// Parts per tile the window split may use for a job (1: never split);
// TcArgs.wsplit and the part-list room follow it.
int tc_window_split(const Geom& g);
// Column parts of the job's class (1: none).  Above 1 the job always runs
// split in that many parts and needs the part-list room.
int tc_column_parts(const Geom& g);
// Shape of the tensor-core geometry a job gets (column parts, A in tensor
// memory, tile slots, tile rows x columns, candidate columns per MMA,
// append-buffer entries); false if the job runs on the direct kernel.
struct TcShape {
    int xs, ts, ns, ty, tx, kcols, kbuf;
};
bool tc_shape(const Geom& g, TcShape& s);

// (a6) float32 boundary re-rank: direct recomputation of the pool's band,
// FP64 only for ties at the K-th boundary; writes the final outputs.
cudaError_t launch_rerank(const Geom& g, const float* img, const float* nrm,
                          const int32_t* pool_idx, const float* pool_score,
                          int32_t* out_idx, float* out_dist, unsigned long long* counters,
                          cudaStream_t st);
struct RerankArgs {
    const float* img;
    const float* nrm;
    const int32_t* pool_idx;
    const float* pool_score;
    int32_t* out_idx;
    float* out_dist;
};
// Jobs that can share one re-rank launch.
bool rerank_same_class(const Geom& a, const Geom& b);
// Several float32 jobs; consecutive jobs of one class share a launch (up to
// 64 each); *nlaunch (nullable) = kernel launches made.
cudaError_t launch_rerank_batch(const Geom* gs, const RerankArgs* as, int n,
                                unsigned long long* counters, cudaStream_t st,
                                int* nlaunch = nullptr);

// Sets the calling thread's bm_last_error message and returns code.
int set_error(int code, const char* msg);
// Text of a timeout code (0x100 + wait site) written by the tensor-core
// kernel's abort path; static storage.
const char* timeout_message(int code);

// (f1) patch groups and reconstruction (groups.cu).
// groups[pt][u][v*C + c] = img[y + u][x + v][c] for idx[pt] = y*W + x (pt =
// r*K + k); a patch whose index is not a top-left of the candidate grid is 0.
cudaError_t launch_gather_groups(const void* img, int dtype, const int32_t* idx, void* out,
                                 int n_ry, int n_rx, int K, int H, int W, int C, int p,
                                 cudaStream_t st);
// out = sum w Z / sum w over the patches deposited at idx (wsum receives the
// per-pixel sum of weights; 0 where none): zeroes both, accumulates, divides.
cudaError_t launch_aggregate(const float* groups, const int32_t* idx, const float* weights,
                             int n_ry, int n_rx, int K, int H, int W, int C, int p, float* out,
                             float* wsum, cudaStream_t st);

}  // namespace bm
