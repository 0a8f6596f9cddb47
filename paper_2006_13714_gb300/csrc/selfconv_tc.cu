// selfconv_tc.cu -- (a3)-(a5): tcgen05 Self-Convolution cross term with the
// distance assembly and the per-reference top-K fused into the epilogue.
//
// What one tile computes.  128 reference patches (a ty x tx block of the
// stride-s reference grid).  For every candidate j in the union of their
// search windows the tensor cores produce, per reference r,
//
//   v(r, j) = <X_r, X_j> - c * n_j          (n_j = ||X_j||^2, the box filter)
//
// i.e. the Self-Convolution C_r(j) of Eq. eq:selfConv (window-restricted as
// in the footnote to Eq. eq:unifySelfConv, summed over channels as S(.) in
// Eq. equ:self-convMM) minus the norm term, which is Theorem 1's
// b = vec(C_r) - 0.5 h_X (.) h_X: the K largest entries of b are the K
// nearest candidates, and d = ||X_r||^2 - 2 b (Lemma 2).  The norm term is an
// extra K-step of the same MMA (A = constant coefficients, B = n_j split into
// three bf16 pieces, precomputed by the box filter), so TMEM already holds
// the score.
//
//   uint8 : operands are centred (x - 128) and A is doubled, all exact in
//           bf16; products and every partial sum are integers below 2^24
//           (p*p*C <= 256), so the FP32 accumulation is exact in any order.
//           The norm K-step uses coefficient -1, so TMEM holds the exact
//           integer v = 2 <X_r, X_j> - n_j and d = n_r - v.
//           Output: the final K (index, distance) per reference.
//   float32: x = hi + lo (bf16 each); cross term = hi.hi + hi.lo + lo.hi; norm
//           coefficient -0.5 plus +eps on a second copy of the pieces, so
//           v = b~ + eps n_j and v + eps n_r bounds the true score from above
//           (|b~ - b| <= eps (n_r + n_j), eps = 2^-14).  Output: a pool of the
//           L largest v per reference for the boundary re-rank kernel.
//
// Data movement (no im2col in HBM).  Per tile, TMA (cp.async.bulk.tensor)
// stages the image tile plus its window halo -- the union of the tile's
// candidate patches -- from each bf16 plane into shared memory.  The
// references' A operand (K-major, canonical no-swizzle core-matrix layout)
// is cut from that staged tile.  Candidates are formed in place, per chunk
// of candidate columns, as "column strips": for candidate column j and
// 16-byte chunk q of a patch row, strip[q][j][row] holds the 8 elements
// starting at pixel (X0 + j) of image row (Y0 + row).  Candidate
// n = j * Rb + row (column-major) then reads patch row u at
// strip[q][j][row + u]: eight consecutive candidates are eight consecutive
// 16-byte rows -- a no-swizzle K-major core matrix -- so every K-step is a
// plain descriptor with SBO = 128 B and LBO = 16 B (next patch row) or the
// q-strip pitch (next chunk of the same row).  The split norms of a chunk's
// columns arrive by bulk copy (cp.async.bulk), one contiguous column each.
//
// Slots.  A CTA keeps NS tiles in flight.  Slot k owns epilogue warps
// 4k..4k+3 (warp 4k+i reads TMEM lanes 32i..32i+31), one producer warp (TMA
// issue, operand formation), one MMA warp (single-thread MMA issue), its own
// shared-memory regions and two TMEM accumulators, so the slots never wait
// on each other; they share only the tensor core.  Every wait is bounded; on
// timeout the CTA sets *status, waits for its copies and MMAs in flight,
// frees its TMEM and returns.
#include "bm_internal.h"

#include <cuda.h>
#include <algorithm>
#include <cuda_bf16.h>

namespace bm {
namespace {

constexpr int kTmemCols = 512;
constexpr float kEps = 6.103515625e-05f;  // 2^-14
constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kSmemLimit = 227 * 1024;
constexpr int kBatch = 8;  // keys merged into the register list at a time
constexpr int kMergeAt = 12;  // merge once a lane holds this many pending keys
constexpr int kMaxSt = 3;  // stages per slot (upper bound)

// Threads of a CTA with NS slots: 4 epilogue warps, 1 producer warp and 1
// MMA warp per slot.
__host__ __device__ constexpr int cta_threads(int ns) { return ns * 192; }

// Class-wide geometry of one launch (every job shares patch, window, stride,
// K, channel padding and dtype; image sizes are per job).
struct TcGeom {
    int Cp, p, h, s, K, HL;
    int rr, rc, wgx, ty, tx;  // lane -> reference mapping and tile shape (references)
    int pw, p_eff, nkc, Rb, kcols;
    int nslots, bufcols, nst; // tiles in flight, TMEM columns per accumulator, stages per slot
    int kbuf;                 // append-buffer entries per lane
    int tbits;                // float32 32-bit keys: window-index bits (0: 64-bit keys)
    int nc_box, base_pitch, base_bytes;  // staged tile: 16-byte chunks per row, row pitch, bytes per plane
    int qpitch, plane_stage, stage_bytes;
    int f32;
    int a_bytes;
    int ts, a_cols;           // A operand in tensor memory (TS MMAs): columns per slot (0: SS)
    int ncc, off_g;           // NCC scores: per-warp 1 / ||X_j|| rows of a column (slot offset)
    int xs;                   // column parts: each part of a tile's candidate columns stages
                              //   only its own columns (1: the whole union in one tile)
    int off_base, off_a, off_stage, off_buf, slot_bytes;  // inside a slot's region
    int off_slots, off_an, off_heap, off_bar, smem_total;
};

// One image of a launch.
struct TcJob {
    CUtensorMap map[2];       // bf16 planes (hi / exact, lo) as {8 elements, row chunks, rows}
    const uint16_t* plane[2]; // the same planes (A read from global memory with column parts)
    int pitch;                // plane row pitch (elements)
    const uint16_t* nsp;      // split norms [Wc][Hc][8] bf16
    const void* nrm;          // int32 / float32 norms [Hc][Wc]
    int32_t* out_idx;         // uint8: final indices
    int32_t* out_dist;        // uint8: final distances
    int32_t* pool_idx;        // float32: pool
    float* pool_score;
    int* status;              // nullable: the job's error word (timeout code on abort)
    int H, W, n_ry, n_rx, Hc, Wc;
    int tiles_x, tile_begin;  // tiles along x; index of the job's first tile (part)
    int wsplit;               // window split: parts per tile (1: none); part q's lists
                              // are references q * nR .. of the output arrays
};

constexpr int kMaxJobs = 64;  // jobs per launch (kept inline in the kernel parameters)
// Window split: a launch whose tiles number fewer than kSplitTarget (the
// SMs of a GB300) splits each job's windows into up to kMaxSplit parts
// (work items), so that small jobs still occupy every SM.  Each part keeps
// its own list, and a part that starts far from the references' centres
// appends more before its threshold tightens, so the split costs selection
// work: it pays only where SMs would otherwise idle (a 512 x 512 image
// alone, 171 tiles, ran 20 % slower split in two).
constexpr int kSplitTarget = 152;
constexpr int kMaxSplit = 4;
constexpr int kSplitChoices = 3;  // tuner: 1, 2 or 4 parts

struct TcParams {
    TcGeom g;
    int njobs, total_tiles;
    int* fault;   // nullable: sticky copy of the first timeout code (context-wide)
    int inject;   // test hook: CTA 0's first producer skips publishing its first stage
    TcJob jobs[kMaxJobs];
};
static_assert(sizeof(TcParams) <= 32764, "kernel parameters exceed the 32 KB limit");

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// try_wait with a suspend-time hint (ns): the waiting thread sleeps until the
// phase completes or the hint elapses instead of spinning on the barrier.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}
// Bounded wait on one mbarrier phase.  False on timeout or abort.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait_sleep(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = code;
            return false;
        }
    }
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The same with A in tensor memory (a_taddr: its first column, lane 0).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d, uint32_t a_taddr, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a_taddr), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 4 consecutive 32-bit columns of the warp's 32 lanes (one value per lane and column).
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
// 32 lanes x (16 * NB) columns: NB aligned x16 loads at taddr + 16*b, one wait.
template <int NB>
__device__ __forceinline__ void tmem_ld_blocks(uint32_t taddr, float* v);
template <>
__device__ __forceinline__ void tmem_ld_blocks<1>(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + 0u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same 16 columns with their maximum per lane (tcgen05.ld.red: the
// load and the reduction in one instruction).
__device__ __forceinline__ void tmem_ld_max(uint32_t taddr, float* v, float& vmax) {
    uint32_t r[16], m;
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %16, [%17];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(m)
        : "r"(taddr + 0u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
    vmax = __uint_as_float(m);
}

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout.
// LBO = byte step between K-adjacent core matrices, SBO = between M/N-adjacent.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint16_t b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
}
__device__ __forceinline__ unsigned orderable(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_orderable(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// TMA: 3-D tiled tensor load global -> shared, completion on an mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
// Bulk (non-tensor) copy global -> shared; 16-byte aligned, size % 16 == 0.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// The 16 bytes starting sh bf16 elements into the 32 bytes {A, B}.
__device__ __forceinline__ uint4 shifted16(const uint4& A, const uint4& B, int sh) {
    const uint32_t w[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
    const int j = sh >> 1;
    uint32_t v[5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
        v[i] = j == 0 ? w[i] : j == 1 ? w[i + 1] : j == 2 ? w[i + 2] : w[i + 3];
    const uint32_t f = (sh & 1) * 16;
    return make_uint4(__funnelshift_r(v[0], v[1], f), __funnelshift_r(v[1], v[2], f),
                      __funnelshift_r(v[2], v[3], f), __funnelshift_r(v[3], v[4], f));
}
// 16 bytes of a staged row starting at element e (any alignment; per-lane e).
__device__ __forceinline__ uint4 lds_shifted16(const uint8_t* row, int e) {
    const uint4* s = reinterpret_cast<const uint4*>(row + (e >> 3) * 16);
    const int sh = e & 7;
    return sh == 0 ? s[0] : shifted16(s[0], s[1], sh);
}
// The same from a plane row in global memory (16-byte aligned rows; the
// plane pitch leaves room for the second chunk).
__device__ __forceinline__ uint4 ldg_shifted16(const uint16_t* row, int e) {
    const uint4* s = reinterpret_cast<const uint4*>(row + (e & ~7));
    const int sh = e & 7;
    const uint4 A = __ldg(s);
    return sh == 0 ? A : shifted16(A, __ldg(s + 1), sh);
}

// Words J .. J+3 of the 32 bytes {a, b}, each shifted right by f bits
// (0 or 16): 16 bytes starting 2J + f/16 bf16 elements in.
template <int J>
__device__ __forceinline__ uint4 shift_pair(const uint4& a, const uint4& b, uint32_t f) {
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    return make_uint4(__funnelshift_r(w[J], w[J + 1], f), __funnelshift_r(w[J + 1], w[J + 2], f),
                      __funnelshift_r(w[J + 2], w[J + 3], f), __funnelshift_r(w[J + 3], w[J + 4], f));
}

// Column strips of NP planes at once: strip row `row` (rows lane, lane + 32,
// ... < Rb) of plane pl = the 16 bytes of staged row `row` starting 2J + f/16
// elements past src[pl] (the same shift for every row).  Two rows per lane
// and every plane in flight per step.
template <int J, int NP>
__device__ __forceinline__ void copy_strips_j(const uint8_t* const (&src)[2], uint8_t* const (&dst)[2],
                                              int pitch, int Rb, int lane, uint32_t f) {
    for (int r0 = 0; r0 < Rb; r0 += 64) {
        uint4 a[NP][2], b[NP][2];
#pragma unroll
        for (int pl = 0; pl < NP; ++pl)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int row = r0 + lane + 32 * t;
                if (row < Rb) {
                    const uint4* sp = reinterpret_cast<const uint4*>(src[pl] + row * pitch);
                    a[pl][t] = sp[0];
                    b[pl][t] = sp[1];
                }
            }
#pragma unroll
        for (int pl = 0; pl < NP; ++pl)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int row = r0 + lane + 32 * t;
                if (row < Rb)
                    *reinterpret_cast<uint4*>(dst[pl] + row * 16) = shift_pair<J>(a[pl][t], b[pl][t], f);
            }
    }
}

// Element shift sh (0..7) of a strip: word offset sh / 2 (compile-time
// case), half-word funnel shift (sh & 1) * 16 bits (run time).
template <int NP>
__device__ __forceinline__ void copy_strips(int sh, const uint8_t* const (&src)[2],
                                            uint8_t* const (&dst)[2], int pitch, int Rb, int lane) {
    const uint32_t f = (uint32_t)(sh & 1) * 16u;
    switch (sh >> 1) {
        case 0: copy_strips_j<0, NP>(src, dst, pitch, Rb, lane, f); break;
        case 1: copy_strips_j<1, NP>(src, dst, pitch, Rb, lane, f); break;
        case 2: copy_strips_j<2, NP>(src, dst, pitch, Rb, lane, f); break;
        default: copy_strips_j<3, NP>(src, dst, pitch, Rb, lane, f); break;
    }
}

// 4-ary max-heap of u64 keys per epilogue thread, element i at h[i * 128]
// (the four children of a node are loaded together: half the dependent
// shared-memory round trips of a binary heap).
struct Heap {
    unsigned long long* h;
    int n;
    __device__ __forceinline__ unsigned long long top() const { return h[0]; }
    __device__ void replace_top(unsigned long long key) {
        int i = 0;
        while (true) {
            const int c0 = 4 * i + 1;
            if (c0 >= n) break;
            unsigned long long cv = h[c0 * 128];
            int c = c0;
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const int ck = c0 + k;
                const unsigned long long v = ck < n ? h[ck * 128] : 0ull;
                if (v > cv) { cv = v; c = ck; }
            }
            if (cv <= key) break;
            h[i * 128] = cv;
            i = c;
        }
        h[i * 128] = key;
    }
    // Sort ascending in place (heap sort).
    __device__ void sort() {
        const int n0 = n;
        for (int m = n0 - 1; m > 0; --m) {
            unsigned long long mx = h[0];
            unsigned long long last = h[m * 128];
            h[m * 128] = mx;
            n = m;
            replace_top(last);
        }
        n = n0;
    }
};

// The same heap with 32-bit keys (float32 pools over 32 entries whose
// window index fits the key's low bits): half the shared memory and traffic.
struct Heap32 {
    unsigned* h;
    int n;
    __device__ __forceinline__ unsigned top() const { return h[0]; }
    __device__ void replace_top(unsigned key) {
        int i = 0;
        while (true) {
            const int c0 = 4 * i + 1;
            if (c0 >= n) break;
            unsigned cv = h[c0 * 128];
            int c = c0;
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const int ck = c0 + k;
                const unsigned v = ck < n ? h[ck * 128] : 0u;
                if (v > cv) { cv = v; c = ck; }
            }
            if (cv <= key) break;
            h[i * 128] = cv;
            i = c;
        }
        h[i * 128] = key;
    }
    __device__ void sort() {
        const int n0 = n;
        for (int m = n0 - 1; m > 0; --m) {
            const unsigned mx = h[0], last = h[m * 128];
            h[m * 128] = mx;
            n = m;
            replace_top(last);
        }
        n = n0;
    }
};

// Compare-exchange: x <- min, y <- max.
__device__ __forceinline__ void cmpx(unsigned long long& x, unsigned long long& y) {
    const bool s = y < x;
    const unsigned long long lo = s ? y : x, hi = s ? x : y;
    x = lo;
    y = hi;
}
__device__ __forceinline__ void cmpx(unsigned& x, unsigned& y) {
    const unsigned lo = min(x, y), hi = max(x, y);
    x = lo;
    y = hi;
}
// Bitonic sort of N registers, ascending.
template <int N, class T>
__device__ __forceinline__ void bitonic_sort(T (&v)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    if ((i & k) == 0) cmpx(v[i], v[l]);
                    else cmpx(v[l], v[i]);
                }
            }
}
// Sort a bitonic sequence of N registers, ascending.
template <int N, class T>
__device__ __forceinline__ void bitonic_merge(T (&v)[N]) {
#pragma unroll
    for (int j = N >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int l = i ^ j;
            if (l > i) cmpx(v[i], v[l]);
        }
}

// Register-resident sorted list (ascending) of the LC best keys.  New keys
// arrive in batches of kBatch: the batch is bitonic-sorted, the LC smallest
// of list + batch are min(a[i], batch[LC-1-i]) (a bitonic sequence), and one
// bitonic merge restores the order -- far fewer compare-exchanges per key
// than a full insertion pass per key.  LC = 24 (not a power of two) runs
// the 32-wide bitonic merge of list ++ reversed batch with the comparators
// that cannot change the 24 smallest left out.  Entries 0..cap-1 are the
// answer (cap <= LC); extra entries only make the list a superset.
template <int LC, class T = unsigned long long>
struct RegTopK {
    T a[LC];
    int cap;
    __device__ __forceinline__ void init(int c) {
        cap = c;
#pragma unroll
        for (int i = 0; i < LC; ++i) a[i] = ~T(0);
    }
    __device__ __forceinline__ void merge_batch(T (&b)[kBatch]) {
        bitonic_sort<kBatch>(b);
        if constexpr (LC == 24) {
            static_assert(kBatch == 8, "the 24-entry merge takes batches of 8");
            // c = a[0..23] ++ (b descending) is bitonic.  Half-cleaner (i, i+16):
            // for i < 8 both are sorted list entries (no exchange); for i >= 8
            // the partner is batch entry 7 - (i - 8)
#pragma unroll
            for (int i = 8; i < 16; ++i) {
                T& hi = b[15 - i];
                const T lo = min(a[i], hi);
                hi = max(a[i], hi);
                a[i] = lo;
            }
            // lower half c[0..15] = a[0..15]: bitonic, sorted by a 16-wide merge;
            // upper half c[16..31] = a[16..23] ++ (b[7..0]): only its 8 smallest
            // are kept -- half-cleaner (16+i, 24+i), then an 8-wide merge
#pragma unroll
            for (int i = 0; i < 8; ++i) a[16 + i] = min(a[16 + i], b[7 - i]);
            T lo16[16], hi8[8];
#pragma unroll
            for (int i = 0; i < 16; ++i) lo16[i] = a[i];
#pragma unroll
            for (int i = 0; i < 8; ++i) hi8[i] = a[16 + i];
            bitonic_merge<16>(lo16);
            bitonic_merge<8>(hi8);
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] = lo16[i];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[16 + i] = hi8[i];
        } else {
#pragma unroll
            for (int i = 0; i < LC; ++i) {
                const int bi = LC - 1 - i;
                if (bi < kBatch) a[i] = b[bi] < a[i] ? b[bi] : a[i];
            }
            bitonic_merge<LC>(a);
        }
    }
    __device__ __forceinline__ T last() const {  // entry cap-1
        if (cap == LC) return a[LC - 1];
        return kth();
    }
    __device__ __forceinline__ T kth() const {  // entry cap-1
        T r = 0;
#pragma unroll
        for (int i = 0; i < LC; ++i) {
            const T x = i < cap ? a[i] : T(0);
            r = x > r ? x : r;
        }
        return r;
    }
};

// float32 pool with 32-bit keys: key = (~orderable(v) with its low tbits
// bits cleared) | window index of the candidate, so one min/max pair is a
// compare-exchange.  The cleared bits round v up by less than 2^tbits ulp
// (v' = from_orderable(~(key & ~M)) >= v); the re-rank widens its band by
// that amount.
template <int LC>
__device__ __forceinline__ void merge_pending32(unsigned* pend, int& cnt, float& thr,
                                                RegTopK<LC, unsigned>& reg, unsigned M) {
    const int m = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
    for (int j0 = 0; j0 < m; j0 += kBatch) {
        unsigned b[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) b[t] = j0 + t < cnt ? pend[(j0 + t) * 128] : ~0u;
        reg.merge_batch(b);
    }
    cnt = 0;
    const unsigned t = reg.last();
    // lowest value whose key can still beat the list's last entry
    if (t != ~0u) thr = from_orderable(~(t | M));
}
template <int LC>
__device__ __noinline__ RegTopK<LC, unsigned> final_merge32(unsigned* pend, int cnt,
                                                            RegTopK<LC, unsigned> reg, unsigned M) {
    float thr = 0.f;
    merge_pending32(pend, cnt, thr, reg, M);
    return reg;
}

// 32-bit pending keys into the lane's shared-memory heap (pools over 32).
__device__ __forceinline__ void merge_pending32_heap(unsigned* pend, int& cnt, float& thr, Heap32& heap,
                                                     unsigned M) {
    for (int j = 0; j < cnt; ++j) {
        const unsigned key = pend[j * 128];
        if (key < heap.top()) heap.replace_top(key);
    }
    cnt = 0;
    const unsigned t = heap.top();
    // lowest value whose key can still beat the heap's worst entry
    if (t != ~0u) thr = from_orderable(~(t | M));
}

// Warp-synchronous merge of every lane's pending entries (call from all 32
// lanes): one pending entry per lane per step goes through the selection.
template <int LC, bool kF32, int PS>
__device__ __forceinline__ void merge_pending(const TcGeom& G, const int* nrm_i, int nr_i,
                                              unsigned long long* pend, int& cnt, float& thr,
                                              RegTopK<LC == 0 ? 1 : LC>& reg, Heap& heap) {
    const int m = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
    for (int j0 = 0; j0 < m; j0 += kBatch) {
        unsigned long long b[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            const int j = j0 + t;
            const unsigned long long e = j < cnt ? pend[j * PS] : kEmpty;
            unsigned long long key = kEmpty;
            if (e != kEmpty) {
                const float v = __uint_as_float((unsigned)(e >> 32));
                const unsigned long long off = e & 0xffffffffull;
                if (kF32) {
                    key = ((unsigned long long)(~orderable(v)) << 32) | off;
                } else {
                    const int dd = nr_i - (int)v;  // v = 2 <X_r, X_j> - ||X_j||^2, exact
                    key = ((unsigned long long)(unsigned)dd << 32) | off;
                }
            }
            b[t] = key;
        }
        if constexpr (LC > 0) {
            reg.merge_batch(b);
        } else {
#pragma unroll 1
            for (int t = 0; t < kBatch; ++t)
                if (b[t] < heap.top()) heap.replace_top(b[t]);
        }
    }
    cnt = 0;
    unsigned long long t;
    if constexpr (LC > 0) t = reg.last();
    else t = heap.top();
    if (t != kEmpty) {
        if (kF32) thr = from_orderable(~(unsigned)(t >> 32));
        else thr = (float)(nr_i - (int)(t >> 32));  // v >= thr  <=>  d <= d_K (exact)
    }
}

// Final flush of the pending entries, out of line (runs once per tile, so
// it stays out of the hot loop's instruction footprint).  The register list
// travels by value.
template <int LC, bool kF32, int PS>
__device__ __noinline__ RegTopK<LC == 0 ? 1 : LC> final_merge(const TcGeom G, const int* nrm_i,
                                                             int nr_i, unsigned long long* pend,
                                                             int cnt, RegTopK<LC == 0 ? 1 : LC> reg,
                                                             unsigned long long* heap_h) {
    float thr = 0.f;
    Heap heap{heap_h, G.HL};
    merge_pending<LC, kF32, PS>(G, nrm_i, nr_i, pend, cnt, thr, reg, heap);
    return reg;
}

// Chunk visiting order: centre-first.  Chunk 0 holds the candidate columns
// at the tile's centre, then alternately right and left, so every reference
// sees its nearest (usually best) candidates first and its threshold
// tightens early.
__device__ __forceinline__ int chunk_order(int c, int n, int cc) {
    const int left = cc, right = n - 1 - cc, m = min(left, right);
    if (c <= 2 * m) {
        const int k = (c + 1) >> 1;
        return (c & 1) ? cc + k : cc - k;
    }
    const int rest = c - 2 * m;
    return left > right ? cc - m - rest : cc + m + rest;
}

// ---------------------------------------------------------------- tiles

struct TileInfo {
    const TcJob* job;
    int ry0, rx0, ry_last, rx_last;
    int Y0, X0, NR, NX, nchunks, center_chunk;
    int part, c0, c1;  // window split: this part's chunks [c0, c1) of the visiting order
                       // (column parts: positional chunks [c0, c1))
    int xs0, pc;       // column parts: first staged candidate column (from X0), and the
                       // chunk the part visits first (relative to c0); 0 otherwise
};

// Work item t of the launch: its job (binary search over the jobs' first
// items), its tile, the union of the tile's references' clipped windows,
// and -- when the job's windows are split -- the part of that union's
// candidate columns this item covers (chunks [c0, c1) of the visiting order;
// the parts of a tile are consecutive items, so they land on different CTAs).
__device__ __forceinline__ TileInfo tile_info(const TcParams& P, int t) {
    const TcGeom& G = P.g;
    int lo = 0, hi = P.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.jobs[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    TileInfo T;
    T.job = &P.jobs[lo];
    const TcJob& J = *T.job;
    const int li = t - J.tile_begin;
    const int lt = li / J.wsplit;
    T.part = li - lt * J.wsplit;
    T.ry0 = (lt / J.tiles_x) * G.ty;
    T.rx0 = (lt % J.tiles_x) * G.tx;
    T.ry_last = min(T.ry0 + G.ty - 1, J.n_ry - 1);
    T.rx_last = min(T.rx0 + G.tx - 1, J.n_rx - 1);
    T.Y0 = max(0, T.ry0 * G.s - G.h);
    const int Y1 = min(J.Hc - 1, T.ry_last * G.s + G.h);
    T.X0 = max(0, T.rx0 * G.s - G.h);
    const int X1 = min(J.Wc - 1, T.rx_last * G.s + G.h);
    T.NR = Y1 - T.Y0 + 1;
    T.NX = X1 - T.X0 + 1;
    T.nchunks = (T.NX + G.kcols - 1) / G.kcols;
    T.center_chunk = min(T.nchunks - 1, ((T.rx0 + T.rx_last) * G.s / 2 - T.X0) / G.kcols);
    T.c0 = T.part * T.nchunks / J.wsplit;
    T.c1 = (T.part + 1) * T.nchunks / J.wsplit;
    T.xs0 = 0;
    T.pc = 0;
    if (G.xs > 1) {
        // column parts: contiguous chunks, visited from the one nearest the
        // tile's centre outwards; the part's staged tile starts at its first
        T.xs0 = T.c0 * G.kcols;
        T.pc = max(0, min(T.center_chunk, T.c1 - 1) - T.c0);
    }
    return T;
}

// Chunk (in column order) of the c-th step of a tile's visiting order.
__device__ __forceinline__ int chunk_at(const TcGeom& G, const TileInfo& T, int c) {
    return G.xs > 1 ? T.c0 + chunk_order(c - T.c0, T.c1 - T.c0, T.pc)
                    : chunk_order(c, T.nchunks, T.center_chunk);
}

// Tile of slot k's g-th turn in CTA b (static round robin over the launch).
__device__ __forceinline__ int slot_tile(int b, int g, int k, int nslots, int grid) {
    return b + (g * nslots + k) * grid;
}

// Barriers of one slot (index into the slot's block of kBarsPerSlot).
enum : int {
    kBarBase = 0,                 // staged tile landed (TMA, tx count)
    kBarAEmpty = 1,               // MMAs of the previous tile done with A
    kBarDone = 2,                 // drain: every MMA of the slot finished
    kBarTFull = 3,                // [2] accumulator ready for the epilogue
    kBarTEmpty = 5,               // [2] accumulator drained by the epilogue (128 arrivals)
    kBarSEmpty = 7,               // [kMaxSt] stage free (MMAs done reading it)
    kBarFull = 7 + kMaxSt,        // [kMaxSt] stage filled: strips formed (producer
                                  //   arrival) and split norms landed (bulk copy, tx count)
    kBarAFull = 7 + 2 * kMaxSt,   // A of the slot's current tile formed (producer)
    kBarsPerSlot = 8 + 2 * kMaxSt
};

// Bounded wait that ignores the abort flag (draining copies in flight).
__device__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity) && globaltimer() - t0 < kWaitNs) {
    }
}

// A operand of a tile: reference patch rows cut from the staged tile, in the
// canonical K-major core-matrix layout (reference m, 16-byte K chunk
// kc = patch row u * pw + chunk q).  Shared by `nparts` threads; this one
// takes items part, part + nparts, ...  uint8: A = 2 (x - 128), exact in
// bf16, so the MMA gives 2 <X_r, X_j>.
template <bool kF32>
__device__ __forceinline__ void form_A(const TcGeom& G, const TileInfo& T, const TcJob& J,
                                       const uint8_t* sbase, uint8_t* sa, int delta, int part,
                                       int nparts) {
    constexpr int nplanes = kF32 ? 2 : 1;
    const int per_m = nplanes * G.nkc;
    const int items = 128 * per_m;
    for (int it = part; it < items; it += nparts) {
        const int m = it / per_m, r = it - m * per_m;
        const int pl = r / G.nkc, kc = r - pl * G.nkc;
        const int u = kc / G.pw, q = kc - u * G.pw;
        const int mw = m >> 5, ml = m & 31;
        const int ry = T.ry0 + (mw / G.wgx) * G.rr + ml / G.rc;
        const int rx = T.rx0 + (mw % G.wgx) * G.rc + ml % G.rc;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (ry < J.n_ry && rx < J.n_rx && u < G.p) {
            const uint8_t* row = sbase + pl * G.base_bytes + (ry * G.s - T.Y0 + u) * G.base_pitch;
            v = lds_shifted16(row, delta + (rx * G.s - T.X0) * G.Cp + 8 * q);
            // zero the elements beyond the patch row (p * Cp elements)
            const int valid = G.p * G.Cp - 8 * q;
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (2 * i >= valid) w[i] = 0;
                else if (2 * i + 1 >= valid) w[i] &= 0xffffu;
                if (!kF32) {
                    const float lo_f = 2.0f * bf16_val((uint16_t)(w[i] & 0xffffu));
                    const float hi_f = 2.0f * bf16_val((uint16_t)(w[i] >> 16));
                    w[i] = (uint32_t)bf16_bits(lo_f) | ((uint32_t)bf16_bits(hi_f) << 16);
                }
            }
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4*>(sa + pl * G.a_bytes + (m >> 3) * G.nkc * 128 + kc * 128 +
                                  (m & 7) * 16) = v;
    }
}

// A in tensor memory, for the TS form of the MMAs (classes whose A operand
// does not fit in shared memory beside the staged tile): each epilogue lane
// writes its own row (TMEM lane m = A row m = reference m of the tile), the
// K elements two per 32-bit column -- 16-byte chunk kc of plane pl at
// columns a_row + (pl * nkc + kc) * 4.  The same values as form_A.  With
// column parts the staged tile need not hold the references' columns, and
// the rows come from the planes in global memory instead.
template <bool kF32>
__device__ __forceinline__ void form_A_tmem(const TcGeom& G, const TileInfo& T, const TcJob& J,
                                            const uint8_t* sbase, int delta, uint32_t a_row, int m) {
    constexpr int nplanes = kF32 ? 2 : 1;
    const int mw = m >> 5, ml = m & 31;
    const int ry = T.ry0 + (mw / G.wgx) * G.rr + ml / G.rc;
    const int rx = T.rx0 + (mw % G.wgx) * G.rc + ml % G.rc;
    const bool ok = ry < J.n_ry && rx < J.n_rx;
    for (int pl = 0; pl < nplanes; ++pl) {
        for (int kc = 0; kc < G.nkc; ++kc) {  // warp-uniform: every lane stores every chunk
            const int u = kc / G.pw, q = kc - u * G.pw;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (ok && u < G.p) {
                if (G.xs > 1) {
                    v = ldg_shifted16(J.plane[pl] + (size_t)(ry * G.s + u) * J.pitch,
                                      rx * G.s * G.Cp + 8 * q);
                } else {
                    const uint8_t* row = sbase + pl * G.base_bytes + (ry * G.s - T.Y0 + u) * G.base_pitch;
                    v = lds_shifted16(row, delta + (rx * G.s - T.X0) * G.Cp + 8 * q);
                }
                const int valid = G.p * G.Cp - 8 * q;
                uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (2 * i >= valid) w[i] = 0;
                    else if (2 * i + 1 >= valid) w[i] &= 0xffffu;
                    if (!kF32) {
                        const float lo_f = 2.0f * bf16_val((uint16_t)(w[i] & 0xffffu));
                        const float hi_f = 2.0f * bf16_val((uint16_t)(w[i] >> 16));
                        w[i] = (uint32_t)bf16_bits(lo_f) | ((uint32_t)bf16_bits(hi_f) << 16);
                    }
                }
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
            tmem_st4(a_row + (uint32_t)((pl * G.nkc + kc) * 4), v);
        }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- the kernel
//
// Persistent: CTA b walks the tiles b, b + G, b + 2G, ... of every job of
// the launch, NS tiles in flight (slot k takes turns k, k + NS, ...).
template <int LC, bool F32, int NS, bool K32>
__global__ void __launch_bounds__(cta_threads(NS), 1)
tc_match_kernel(const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcGeom& G = P.g;
    constexpr bool kF32 = F32;
    constexpr int kEpiWarps = 4 * NS;
    constexpr int kThreads = cta_threads(NS);
    constexpr int nplanes = kF32 ? 2 : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grid = gridDim.x, cta = blockIdx.x;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G.off_bar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NS * kBarsPerSlot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar0 = smem_u32(bars);
    auto BAR = [bar0](int k, int i) -> uint32_t { return bar0 + 8u * (uint32_t)(k * kBarsPerSlot + i); };

    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) {
            mbar_init(BAR(k, kBarBase), 1);
            mbar_init(BAR(k, kBarAEmpty), 1);
            mbar_init(BAR(k, kBarDone), 1);
            for (int b = 0; b < 2; ++b) {
                mbar_init(BAR(k, kBarTFull + b), 1);
                mbar_init(BAR(k, kBarTEmpty + b), 128);
            }
            for (int i = 0; i < kMaxSt; ++i) {
                mbar_init(BAR(k, kBarSEmpty + i), 1);
                mbar_init(BAR(k, kBarFull + i), 1);
            }
            mbar_init(BAR(k, kBarAFull), 5);  // 4 epilogue warps + the producer
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    constexpr int kMmaWarp0 = kEpiWarps + NS;  // MMA warp of slot k: kMmaWarp0 + k
    if (warp == kMmaWarp0) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    // A_norm (shared by all tiles): [group][2 kchunks][8 x 16 B], the
    // coefficients of the norm pieces
    for (int t = threadIdx.x; t < 128 * 2; t += kThreads) {
        const int m = t >> 1, kc = t & 1;
        uint16_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (kc == 0) {
            const uint16_t cn = bf16_bits(kF32 ? -0.5f : -1.0f);
            c[0] = c[1] = c[2] = cn;
            if (kF32) c[3] = c[4] = c[5] = bf16_bits(kEps);
        }
        const uint4 val = make_uint4(c[0] | (uint32_t(c[1]) << 16), c[2] | (uint32_t(c[3]) << 16),
                                     c[4] | (uint32_t(c[5]) << 16), c[6] | (uint32_t(c[7]) << 16));
        *reinterpret_cast<uint4*>(smem + G.off_an + (m >> 3) * 256 + kc * 128 + (m & 7) * 16) = val;
    }
    // stages start zeroed: rows no copy writes stay finite
    for (int k = 0; k < NS; ++k)
        for (int t = threadIdx.x; t < G.nst * G.stage_bytes / 16; t += kThreads)
            reinterpret_cast<uint4*>(smem + G.off_slots + k * G.slot_bytes + G.off_stage)[t] =
                make_uint4(0, 0, 0, 0);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp >= kEpiWarps && warp < kMmaWarp0) {
        // ------------------------------------------------------------ producer warp of slot k
        const int k = warp - kEpiWarps;
        uint8_t* slot = smem + G.off_slots + k * G.slot_bytes;
        uint8_t* sbase = slot + G.off_base;
        uint8_t* sa = slot + G.off_a;
        const uint32_t box_bytes = (uint32_t)G.nc_box * 16u * (uint32_t)G.Rb;
        int base_pending = -1;  // staged-tile copy in flight (drained on abort)
        int cs = 0;             // slot-local chunk counter: stage ring
        bool ok = true;
        for (int turn = 0; ok && !*abort_flag; ++turn) {
            const int tile = slot_tile(cta, turn, k, NS, grid);
            if (tile >= P.total_tiles) break;
            const TileInfo T = tile_info(P, tile);
            const TcJob& J = *T.job;
            // (column parts: the staged tile starts at the part's first column)
            const int xst = (T.X0 + T.xs0) * G.Cp;
            const int e0 = xst & ~7, delta = xst - e0;
            // (1) stage the tile plus halo: this warp is done reading the
            // previous one, and the epilogue warps are once the previous A is formed
            if (turn > 0 && !__all_sync(0xffffffffu, mbar_wait(BAR(k, kBarAFull), (turn - 1) & 1, abort_flag, 7)))
                break;
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_expect_tx(BAR(k, kBarBase), nplanes * box_bytes);
                for (int pl = 0; pl < nplanes; ++pl)
                    tma_load_3d(smem_u32(sbase + pl * G.base_bytes), &J.map[pl], 0, e0 >> 3, T.Y0,
                                BAR(k, kBarBase));
            }
            base_pending = turn & 1;
            // (2) A region free (previous tile's MMAs done) and the tile landed
            if (turn > 0) ok = __all_sync(0xffffffffu, mbar_wait(BAR(k, kBarAEmpty), (turn - 1) & 1, abort_flag, 5));
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(BAR(k, kBarBase), turn & 1, abort_flag, 6));
            if (!ok) break;
            base_pending = -1;
            // (3) this warp's share of A (the slot's epilogue warps form the rest;
            // with A in tensor memory they form all of it)
            if (!G.ts) form_A<kF32>(G, T, J, sbase, sa, delta, 128 + lane, 160);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(BAR(k, kBarAFull));
            // (4) chunks: stage free -> split norms by bulk copy -> strips
            // formed in place -> arrival on the stage's barrier
            const int rows = min(G.Rb, J.Hc - T.Y0);
            for (int c = T.c0; c < T.c1; ++c, ++cs) {
                const int stage = cs % G.nst, use = cs / G.nst;
                if (use > 0 && !__all_sync(0xffffffffu, mbar_wait(BAR(k, kBarSEmpty + stage), (use - 1) & 1, abort_flag, 1))) {
                    ok = false;
                    break;
                }
                uint8_t* sb = slot + G.off_stage + stage * G.stage_bytes;
                const int jc0 = chunk_at(G, T, c) * G.kcols;
                const int kc_here = min(G.kcols, T.NX - jc0);
                if (lane == 0) {
                    uint8_t* nsb = sb + nplanes * G.plane_stage;
                    mbar_expect_tx(BAR(k, kBarFull + stage), (uint32_t)(kc_here * rows * 16));
                    for (int jl = 0; jl < kc_here; ++jl)
                        bulk_load(smem_u32(nsb + jl * G.Rb * 16),
                                  J.nsp + ((size_t)(T.X0 + jc0 + jl) * J.Hc + T.Y0) * 8,
                                  (uint32_t)(rows * 16), BAR(k, kBarFull + stage));
                }
                for (int q = 0; q < G.pw; ++q)
                    for (int jl = 0; jl < kc_here; ++jl) {
                        const int ecol = delta + (jc0 - T.xs0 + jl) * G.Cp + 8 * q;
                        const uint8_t* const src[2] = {sbase + (ecol >> 3) * 16,
                                                       sbase + G.base_bytes + (ecol >> 3) * 16};
                        uint8_t* const dst[2] = {sb + q * G.qpitch + jl * G.Rb * 16,
                                                 sb + G.plane_stage + q * G.qpitch + jl * G.Rb * 16};
                        copy_strips<nplanes>(ecol & 7, src, dst, G.base_pitch, G.Rb, lane);
                    }
                fence_proxy_async();
                __syncwarp();
                // (the test hook withholds this arrival once: the MMA warp's bounded
                // wait on the stage then runs out and the CTA takes its abort path)
                const bool withhold = P.inject && cta == 0 && k == 0 && turn == 0 && c == T.c0;
                if (lane == 0 && !withhold) mbar_arrive(BAR(k, kBarFull + stage));
            }
        }
        // drain the copies in flight before the shared memory is released:
        // the staged tile, and the split norms of the last use of each stage
        if (lane == 0) {
            if (base_pending >= 0) mbar_drain(BAR(k, kBarBase), base_pending);
            for (int i = 0; i < G.nst && i < cs; ++i) {
                const int csn = cs - 1 - i;
                mbar_drain(BAR(k, kBarFull + csn % G.nst), (csn / G.nst) & 1);
            }
        }
        __syncwarp();
    } else if (warp >= kMmaWarp0) {
        // ------------------------------------------------------------ MMA warp of slot k
        const int k = warp - kMmaWarp0;
        if (lane == 0) {
            uint8_t* slot = smem + G.off_slots + k * G.slot_bytes;
            const uint32_t an = smem_u32(smem + G.off_an);
            const uint32_t sbo_a = G.nkc * 128;
            const uint32_t lbo_b = G.pw == 1 ? 16u : (uint32_t)G.qpitch;
            // descriptors: the start-address field (address >> 4) of a base
            // descriptor plus the operand offset >> 4 (shared-memory addresses
            // stay below 2^18, no carry out of the field)
            const uint64_t da_hi = sdesc(smem_u32(slot + G.off_a), 128, sbo_a);
            const uint64_t da_lo = da_hi + (uint64_t)(G.a_bytes >> 4);
            const uint64_t dn_a = sdesc(an, 128, 256);
            const uint32_t ta_hi = tmem_base + (uint32_t)(2 * NS * G.bufcols + k * G.a_cols);  // TS
            int cs = 0;
            bool ok = true;
            for (int turn = 0; ok; ++turn) {
                const int tile = slot_tile(cta, turn, k, NS, grid);
                if (tile >= P.total_tiles) break;
                const TileInfo T = tile_info(P, tile);
                if (!mbar_wait(BAR(k, kBarAFull), turn & 1, abort_flag, 7)) break;
                if (T.c0 == T.c1) mma_commit(BAR(k, kBarAEmpty));  // a part with no columns
                for (int c = T.c0; c < T.c1; ++c, ++cs) {
                    const int stage = cs % G.nst, use = cs / G.nst;
                    const int buf = cs & 1, ub = cs >> 1;
                    if (ub > 0 && !mbar_wait(BAR(k, kBarTEmpty + buf), (ub - 1) & 1, abort_flag, 2)) {
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(BAR(k, kBarFull + stage), use & 1, abort_flag, 3)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int jc0 = chunk_at(G, T, c) * G.kcols;
                    const int kc_here = min(G.kcols, T.NX - jc0);
                    const uint32_t idesc = idesc_bf16(128, kc_here * G.Rb);
                    const uint32_t d = tmem_base + (2 * k + buf) * G.bufcols;
                    const uint32_t sbu = smem_u32(slot + G.off_stage + stage * G.stage_bytes);
                    const uint64_t db_hi = sdesc(sbu, lbo_b, 128);
                    const uint64_t db_lo = db_hi + (uint64_t)(G.plane_stage >> 4);
                    uint32_t acc = 0;
                    int u = 0, qq = 0;
                    if (G.ts) {
                        // A in tensor memory: K chunks kc, kc + 1 at columns 4 kc ..
                        for (int kc = 0; kc < G.nkc; kc += 2) {
                            const uint64_t ob = (uint64_t)((qq * G.qpitch + u * 16) >> 4);
                            const uint32_t ta = ta_hi + (uint32_t)(kc * 4);
                            mma_bf16_ts(d, ta, db_hi + ob, idesc, acc);
                            acc = 1;
                            if (kF32) {
                                mma_bf16_ts(d, ta, db_lo + ob, idesc, 1);
                                mma_bf16_ts(d, ta + (uint32_t)(G.nkc * 4), db_hi + ob, idesc, 1);
                            }
                            qq += 2;
                            while (qq >= G.pw) { qq -= G.pw; ++u; }
                        }
                    } else {
                        for (int kc = 0; kc < G.nkc; kc += 2) {
                            const uint64_t oa = (uint64_t)(kc * 8);  // kc * 128 bytes
                            const uint64_t ob = (uint64_t)((qq * G.qpitch + u * 16) >> 4);
                            mma_bf16(d, da_hi + oa, db_hi + ob, idesc, acc);
                            acc = 1;
                            if (kF32) {
                                mma_bf16(d, da_hi + oa, db_lo + ob, idesc, 1);
                                mma_bf16(d, da_lo + oa, db_hi + ob, idesc, 1);
                            }
                            // next pair of 16-byte K chunks: (u, q) advances by two in row-major order
                            qq += 2;
                            while (qq >= G.pw) { qq -= G.pw; ++u; }
                        }
                    }
                    // NCC (never 32-bit keys): no norm K-step (the score is scaled in the epilogue)
                    if (K32 || !G.ncc)
                        mma_bf16(d, dn_a, sdesc(sbu + nplanes * G.plane_stage, 16, 128), idesc, 1);
                    mma_commit(BAR(k, kBarSEmpty + stage));
                    mma_commit(BAR(k, kBarTFull + buf));
                    if (c + 1 == T.c1) mma_commit(BAR(k, kBarAEmpty));  // A free once these finish
                }
            }
            // drain: every MMA issued by this thread finishes before TMEM is freed
            mma_commit(BAR(k, kBarDone));
            mbar_drain(BAR(k, kBarDone), 0);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        // Slot k = warp / 4.  Per lane: the best keys of its reference (uint8:
        // (d, offset), float32: (-v, offset)) in a register list (or a shared-
        // memory heap for large K) behind an append buffer: values at or above
        // the lane's threshold are appended with predicated stores; when any
        // lane's buffer nears full the warp merges in lock-step.
        const int k = warp >> 2, quarter = warp & 3;
        uint8_t* slot = smem + G.off_slots + k * G.slot_bytes;
        unsigned long long* pend =
            reinterpret_cast<unsigned long long*>(slot + G.off_buf) + (threadIdx.x & 127);
        unsigned* pend32 = reinterpret_cast<unsigned*>(slot + G.off_buf) + (threadIdx.x & 127);
        const unsigned kM = (1u << G.tbits) - 1u;   // window-index bits of a 32-bit key
        const int ww = 2 * G.h + 1;
        Heap heap{reinterpret_cast<unsigned long long*>(smem + G.off_heap) + (threadIdx.x & 127), G.HL};
        Heap32 heap32{reinterpret_cast<unsigned*>(smem + G.off_heap) + (threadIdx.x & 127), G.HL};
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        int qc = 0;  // slot-local chunk counter (accumulator phase)
        for (int turn = 0; !*abort_flag; ++turn) {
            const int tile = slot_tile(cta, turn, k, NS, grid);
            if (tile >= P.total_tiles) break;
            const TileInfo T = tile_info(P, tile);
            const TcJob& J = *T.job;
            RegTopK<LC == 0 ? 1 : LC> reg;
            RegTopK<(K32 && LC > 0) ? LC : 32, unsigned> reg32;
            if constexpr (K32 && LC > 0) reg32.init(G.HL);
            else if constexpr (LC > 0) reg.init(G.HL);
            if constexpr (LC == 0 && K32) {
                for (int i = 0; i < G.HL; ++i) heap32.h[i * 128] = ~0u;
            } else if constexpr (LC == 0) {
                for (int i = 0; i < G.HL; ++i) heap.h[i * 128] = kEmpty;
            }
            const int ry = T.ry0 + (quarter / G.wgx) * G.rr + lane / G.rc;
            const int rx = T.rx0 + (quarter % G.wgx) * G.rc + lane % G.rc;
            const bool lane_ok = ry < J.n_ry && rx < J.n_rx;
            const int yr = ry * G.s, xr = rx * G.s;
            // this lane's candidate rows inside the strip (empty if no reference)
            const int lo = lane_ok ? max(0, yr - G.h - T.Y0) : 1 << 20;
            const int hi = lane_ok ? min(T.NR - 1, yr + G.h - T.Y0) : -1;
            const int* nrm_i = static_cast<const int*>(J.nrm);
            const int nr_i = (lane_ok && !kF32) ? nrm_i[(size_t)yr * J.Wc + xr] : 0;
            // the slot's A operand (with the producer): the A region is free
            // once the previous tile's MMAs are done, the staged tile has landed
            if (turn > 0 && !mbar_wait(BAR(k, kBarAEmpty), (turn - 1) & 1, abort_flag, 5)) break;
            tc_fence_after();
            if (!mbar_wait(BAR(k, kBarBase), turn & 1, abort_flag, 6)) break;
            {
                const int e0 = (T.X0 * G.Cp) & ~7;
                if (G.ts)
                    form_A_tmem<kF32>(G, T, J, smem + G.off_slots + k * G.slot_bytes + G.off_base,
                                      T.X0 * G.Cp - e0,
                                      tmem_base + lane_base + (uint32_t)(2 * NS * G.bufcols + k * G.a_cols),
                                      threadIdx.x & 127);
                else
                    form_A<kF32>(G, T, J, smem + G.off_slots + k * G.slot_bytes + G.off_base,
                                 smem + G.off_slots + k * G.slot_bytes + G.off_a, T.X0 * G.Cp - e0,
                                 threadIdx.x & 127, 160);
                fence_proxy_async();
                tc_fence_before();  // tensor-memory A: its stores before the MMAs
                __syncwarp();
                if (lane == 0) mbar_arrive(BAR(k, kBarAFull));
            }
            float thr = -__int_as_float(0x7f800000);  // -inf while the list has empty slots
            int cnt = 0;
            const int merge_at = min(kMergeAt, G.kbuf - 15);  // room for one more block
            for (int c = T.c0; c < T.c1; ++c, ++qc) {
                const int buf = qc & 1, ub = qc >> 1;
                if (!mbar_wait(BAR(k, kBarTFull + buf), ub & 1, abort_flag, 4)) break;
                tc_fence_after();
                const int jc0 = chunk_at(G, T, c) * G.kcols;
                const int kc_here = min(G.kcols, T.NX - jc0);
                for (int jl = 0; jl < kc_here; ++jl) {
                    const int xc = T.X0 + jc0 + jl;
                    const bool xok = lane_ok && abs(xc - xr) <= G.h;
                    if (!__any_sync(0xffffffffu, xok)) continue;
                    // rows any lane of the warp needs in this column (warp-uniform)
                    const int wlo = __reduce_min_sync(0xffffffffu, xok ? lo : 1 << 20);
                    const int whi = __reduce_max_sync(0xffffffffu, xok ? hi : -1);
                    const int b0 = wlo >> 4, nblk = (whi >> 4) - b0 + 1;
                    const uint32_t colbase = tmem_base + lane_base + (2 * k + buf) * G.bufcols +
                                             jl * G.Rb + 16 * b0;
                    // NCC: 1 / ||X_j|| of this column's candidate rows, into the warp's
                    // own shared-memory row (read back by broadcast)
                    float* gw = reinterpret_cast<float*>(slot + G.off_g) + quarter * 256;
                    if (!K32 && G.ncc) {
                        const uint4* gsrc = reinterpret_cast<const uint4*>(J.nsp) + (size_t)xc * J.Hc + T.Y0;
                        for (int rr = 16 * b0 + lane; rr < 16 * (b0 + nblk); rr += 32)
                            gw[rr] = T.Y0 + rr < J.Hc ? __uint_as_float(__ldg(&gsrc[rr].x)) : 0.f;
                        __syncwarp();
                    }
                    for (int bb = 0; bb < nblk; ++bb) {
                        float w[16], wmax;
                        tmem_ld_max(colbase + 16 * bb, w, wmax);
                        if (!K32 && G.ncc) {
                            // the score a_j / ||X_j||: the maximum is of the scaled values
                            const float4* g4 = reinterpret_cast<const float4*>(gw + 16 * (b0 + bb));
                            wmax = -__int_as_float(0x7f800000);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float4 gq = g4[q];
                                w[4 * q] *= gq.x; w[4 * q + 1] *= gq.y; w[4 * q + 2] *= gq.z; w[4 * q + 3] *= gq.w;
                            }
#pragma unroll
                            for (int i = 0; i < 16; ++i) wmax = fmaxf(wmax, w[i]);
                        }
                        // a block whose values all fall below every lane's threshold
                        // adds nothing: skipped on the load's own maximum (which also
                        // covers rows outside a lane's window -- a false positive
                        // only costs the full test below)
                        if (!__any_sync(0xffffffffu, xok && wmax >= thr)) continue;
                        const int b = b0 + bb;
                        // this lane's valid rows of block b: [max(i0, 0), min(i1, 15)]
                        const int i0 = max(lo - 16 * b, 0), i1 = min(hi - 16 * b, 15);
                        const unsigned rows = (xok && i1 >= i0)
                                                  ? ((0xffffu >> (15 - i1)) & (0xffffu << i0))
                                                  : 0u;
                        // rows at or above the threshold, as a bit mask
                        unsigned bits = 0;
#pragma unroll
                        for (int i = 0; i < 16; ++i) bits |= (w[i] >= thr ? 1u : 0u) << i;
                        bits &= rows;
                        // append the rows whose bit is set: dense blocks with one
                        // predicated store per row, sparse ones bit by bit (the
                        // row's value picked by a 4-level select tree on its index)
                        const int most = __reduce_max_sync(0xffffffffu, (unsigned)__popc(bits));
                        if (most > 0) {
                            unsigned base;
                            int step;
                            if constexpr (K32) {
                                // window index of row 16b + i: (row - yr + h) * ww + (xc - xr + h)
                                base = (unsigned)((T.Y0 + 16 * b - yr + G.h) * ww + (xc - xr + G.h));
                                step = ww;
                            } else {
                                base = (unsigned)((T.Y0 + 16 * b) * J.W + xc);
                                step = J.W;
                            }
                            auto put = [&](int slot_i, float wi, int i) {
                                if constexpr (K32)
                                    pend32[slot_i * 128] = (~orderable(wi) & ~kM) | (base + (unsigned)(i * step));
                                else
                                    pend[slot_i * 128] = ((unsigned long long)__float_as_uint(wi) << 32) |
                                                         (base + (unsigned)(i * step));
                            };
                            if (most > 4) {
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    if (bits & (1u << i)) put(cnt, w[i], i);
                                    cnt += (bits >> i) & 1u;
                                }
                            } else {
                                while (bits) {
                                    const int i = __ffs(bits) - 1;
                                    bits &= bits - 1;
                                    float s8[8], s4[4], s2[2];
#pragma unroll
                                    for (int t = 0; t < 8; ++t) s8[t] = (i & 1) ? w[2 * t + 1] : w[2 * t];
#pragma unroll
                                    for (int t = 0; t < 4; ++t) s4[t] = (i & 2) ? s8[2 * t + 1] : s8[2 * t];
#pragma unroll
                                    for (int t = 0; t < 2; ++t) s2[t] = (i & 4) ? s4[2 * t + 1] : s4[2 * t];
                                    put(cnt, (i & 8) ? s2[1] : s2[0], i);
                                    ++cnt;
                                }
                            }
                        }
                        // keep room for the next block's appends
                        if (__any_sync(0xffffffffu, cnt >= merge_at)) {
                            if constexpr (K32 && LC == 0) merge_pending32_heap(pend32, cnt, thr, heap32, kM);
                            else if constexpr (K32) merge_pending32(pend32, cnt, thr, reg32, kM);
                            else merge_pending<LC, kF32, 128>(G, nrm_i, nr_i, pend, cnt, thr, reg, heap);
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(BAR(k, kBarTEmpty + buf));
            }
            if (__any_sync(0xffffffffu, cnt > 0)) {
                if constexpr (K32 && LC == 0) {
                    float thr0 = 0.f;
                    merge_pending32_heap(pend32, cnt, thr0, heap32, kM);
                } else if constexpr (K32) reg32 = final_merge32(pend32, cnt, reg32, kM);
                else reg = final_merge<LC, kF32, 128>(G, nrm_i, nr_i, pend, cnt, reg, heap.h);
            }
            // ---- write results
            if (lane_ok && !*abort_flag) {
                // a window part writes its own list (merged by split_merge_kernel)
                const size_t ref = (size_t)ry * J.n_rx + rx + (size_t)T.part * J.n_ry * J.n_rx;
                if constexpr (LC == 0 && K32) heap32.sort();  // outputs and pools best first
                else if constexpr (LC == 0) heap.sort();
                const int nout = kF32 ? G.HL : G.K;
                auto emit = [&](int i, unsigned long long key) {
                    if (kF32) {
                        // pool: best first (the list order)
                        J.pool_idx[ref * G.HL + i] =
                            key == kEmpty ? -1 : (int32_t)(unsigned)(key & 0xffffffffu);
                        J.pool_score[ref * G.HL + i] =
                            key == kEmpty ? -__int_as_float(0x7f800000)
                                          : from_orderable(~(unsigned)(key >> 32));
                    } else {
                        J.out_idx[ref * G.K + i] =
                            key == kEmpty ? -1 : (int32_t)(unsigned)(key & 0xffffffffu);
                        J.out_dist[ref * G.K + i] =
                            key == kEmpty ? 0x7fffffff : (int32_t)(unsigned)(key >> 32);
                    }
                };
                if constexpr (K32) {
                    auto emit32 = [&](int i, unsigned key) {
                        int32_t off = -1;
                        float v = -__int_as_float(0x7f800000);
                        if (key != ~0u) {
                            const int li = (int)(key & kM);
                            const int dy = li / ww - G.h, dx = li % ww - G.h;
                            off = (yr + dy) * J.W + (xr + dx);
                            v = from_orderable(~(key & ~kM));  // upper end of the key's bucket
                        }
                        J.pool_idx[ref * G.HL + i] = off;
                        J.pool_score[ref * G.HL + i] = v;
                    };
                    if constexpr (LC > 0) {
#pragma unroll
                        for (int i = 0; i < LC; ++i)
                            if (i < nout) emit32(i, reg32.a[i]);
                    } else {
                        for (int i = 0; i < nout; ++i) emit32(i, heap32.h[i * 128]);
                    }
                } else if constexpr (LC > 0) {
#pragma unroll
                    for (int i = 0; i < LC; ++i)
                        if (i < nout) emit(i, reg.a[i]);
                } else {
                    for (int i = 0; i < nout; ++i) emit(i, heap.h[i * 128]);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
    // an aborted CTA leaves parts of any job of the launch unwritten: every
    // job's error word gets the timeout code
    if (threadIdx.x == 0 && *abort_flag) {
        for (int j = 0; j < P.njobs; ++j)
            if (P.jobs[j].status) atomicExch(P.jobs[j].status, 0x100 + *abort_flag);
        if (P.fault) atomicCAS(P.fault, 0, 0x100 + *abort_flag);
    }
}

// Class geometry for a job shape: lane mapping, strips, slots, shared memory.
// Preference: two tiles in flight (when the list lives in registers), then
// the mapping with the least MMA work, then the largest append buffer and
// the deepest stage ring that fit the shared memory.  Classes where nothing
// fits split each tile's candidate columns into xs = 2, 3 or 4 contiguous
// parts (separate work items whose lists the split merge joins), each
// staging only its own columns: the staged tile shrinks by about xs, and A
// (in tensor memory) is read from the planes in global memory.
bool make_tc_geom(const Geom& g, TcGeom& t, int choice = -1, int* nchoices = nullptr) {
    t = TcGeom{};
    t.Cp = g.Cp; t.p = g.p; t.h = g.h; t.s = g.s; t.K = g.K;
    t.pw = g.pw; t.p_eff = g.p_eff; t.nkc = g.p_eff * g.pw;
    // NCC keeps a pool by score for both dtypes (the float32 form of the
    // kernel; uint8 operands are exact in its hi plane, its lo plane is 0)
    t.ncc = g.ncc;
    t.f32 = g.dtype == kF32 || g.ncc;
    t.HL = t.f32 ? g.L : g.K;
    const int nplanes = t.f32 ? 2 : 1;
    // float32 lists in registers use 32-bit keys when the window index fits
    // 12 bits (window <= 63): up to 2^(bits-23) relative rounding of the pool
    // scores.  Pools over 32 (the shared-memory heap) keep 64-bit keys when
    // they fit -- the rounding widens the re-rank's band, which for K 70 at
    // window 61 sent a quarter of the references to a window recompute -- and
    // take 32-bit keys (half the heap) when nothing else fits.  Column parts
    // cost selection work (each part fills its own list), so at 11 window-
    // index bits the fewest parts come first whatever the keys; at 12 bits
    // (2^-11 rounding) 64-bit keys come first, with more parts if need be --
    // unless the pool has 24 or more entries beyond K, which absorb the
    // rounding (then the fewest parts come first again).
    // Measured on four-channel float32, K 70 (matching plus re-rank):
    // window 39, one part with 32-bit keys 17.2 M references/s against 14.8
    // for two parts with 64-bit keys; window 61, p 7: three parts with
    // 64-bit keys 7.3 M/s against 6.2 for two parts with 32-bit keys.
    int tb32 = 0;
    if (t.f32 && !t.ncc) {  // NCC: exact scores (its scores cluster near the top)
        const int ww = 2 * g.h + 1;
        int b = 1;
        while ((1 << b) < ww * ww) ++b;
        if (b <= 12) tb32 = b;
    }
    t.tbits = t.HL <= 32 ? tb32 : 0;
    const TcGeom t0 = t;
    const bool keys_first = tb32 >= 12 && g.L - g.K < 24;
    for (int it = 0; it < 2 * kMaxSplit; ++it) {
    const int keys = keys_first ? it / kMaxSplit : it & 1;
    const int xs = keys_first ? it % kMaxSplit + 1 : (it >> 1) + 1;
    if (xs > 1 && t0.ncc) continue;
    t = t0;
    if (keys == 1) {
        if (t.HL <= 32 || !tb32) continue;
        t.tbits = tb32;
    }
    t.xs = xs;
    // lane -> reference mapping: rr reference rows x rc columns per warp, a
    // wgy x wgx grid of 4 warps
    static const int kMaps[6][2] = {{8, 2}, {16, 4}, {32, 4}, {8, 4}, {4, 4}, {1, 1}};
    // A in shared memory first; classes where nothing fits (the staged tile
    // plus A beyond 227 KB: float32 with four channels, large windows) keep
    // A in tensor memory instead (TS MMAs), beside narrower accumulators
    for (int ts = xs > 1 ? 1 : 0; ts <= 1; ++ts)
    for (int ns = 2; ns >= 1; --ns) {
        if (ns == 2 && t.HL > 32) continue;
        const int a_cols = ts ? nplanes * t.nkc * 4 : 0;  // 16-bit elements, two per column
        const int bufcols = ((kTmemCols - ns * a_cols) / (2 * ns)) / 16 * 16;
        if (bufcols < 16) continue;
        bool found = false;
        long long best = 0;
        TcGeom bestc{};
        int ncand = 0;
        for (const auto& mp : kMaps)
            for (int kbuf = 32; kbuf >= 16; kbuf -= 8)
                for (int nst = kMaxSt; nst >= 2; --nst) {
                    TcGeom c = t;
                    const int rr = mp[0], wgx = mp[1], rc = 32 / rr, wgy = 4 / wgx;
                    c.rr = rr; c.rc = rc; c.wgx = wgx; c.ty = wgy * rr; c.tx = wgx * rc;
                    const int nr_max = (c.ty - 1) * g.s + 2 * g.h + 1;
                    const int nx_max = (c.tx - 1) * g.s + 2 * g.h + 1;
                    c.Rb = (nr_max + g.p_eff - 1 + 15) / 16 * 16;
                    if (c.Rb > bufcols) continue;
                    c.kcols = bufcols / c.Rb;
                    // candidate columns one staged tile covers: the union, or
                    // the largest column part of it
                    const int nch = (nx_max + c.kcols - 1) / c.kcols;
                    const int cols = std::min(nx_max, (nch + xs - 1) / xs * c.kcols);
                    // staged row: alignment slack + every candidate column's patch row;
                    // an odd 16-byte chunk count keeps 16-byte row reads conflict-free
                    c.nc_box = ((7 + (cols - 1) * g.Cp + 8 * g.pw + 7) / 8) | 1;
                    if (c.nc_box > 255) continue;
                    c.nslots = ns;
                    c.bufcols = bufcols;
                    c.nst = nst;
                    c.kbuf = kbuf;
                    c.base_pitch = c.nc_box * 16;
                    c.base_bytes = c.Rb * c.base_pitch;
                    c.qpitch = (c.kcols * c.Rb + g.p_eff + 16) * 16;
                    c.plane_stage = c.pw * c.qpitch;
                    c.stage_bytes = (nplanes * c.plane_stage + c.kcols * c.Rb * 16 + 127) / 128 * 128;
                    c.ts = ts;
                    c.a_cols = a_cols;
                    c.a_bytes = ts ? 0 : 128 * c.nkc * 16;
                    // one slot: staged tile, A, stages, append buffers
                    int off = 0;
                    c.off_base = off; off += (nplanes * c.base_bytes + 1023) / 1024 * 1024;
                    c.off_a = off; off += nplanes * c.a_bytes;
                    c.off_stage = off; off += nst * c.stage_bytes;
                    c.off_buf = off; off += 128 * kbuf * (c.tbits ? 4 : 8);  // 32- or 64-bit keys
                    c.off_g = off; off += g.ncc ? 4 * 256 * 4 : 0;  // NCC: a column's 1/||X_j||, per warp
                    c.slot_bytes = (off + 1023) / 1024 * 1024;
                    off = 0;
                    c.off_slots = off; off += ns * c.slot_bytes;
                    c.off_an = off; off += 128 * 2 * 16;
                    c.off_heap = off; off += c.HL > 32 ? 128 * c.HL * (c.tbits ? 4 : 8) : 0;
                    c.off_bar = off; off += ns * kBarsPerSlot * 8 + 16;
                    c.smem_total = (off + 1023) / 1024 * 1024;
                    if (c.smem_total > kSmemLimit) continue;
                    // an explicit choice (autotuner) is the choice-th fitting candidate
                    if (ncand++ == choice) {
                        t = c;
                        if (nchoices) *nchoices = -1;  // counting stops at the pick
                        return true;
                    }
                    // least MMA work (union columns x strip rows); among equals the
                    // first fit: the larger append buffer, then deeper stages
                    const long long work = (long long)nx_max * c.Rb;
                    if (!found || work < best) {
                        found = true;
                        best = work;
                        bestc = c;
                    }
                }
        if (found) {
            if (nchoices) *nchoices = ncand;
            if (choice >= ncand) return false;  // no such candidate
            t = bestc;
            return true;
        }
    }
    }  // (keys, xs)
    return false;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the CUDA runtime).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Plane as a 3-D tensor {8 elements, 16-byte chunks of a row, rows}; the box
// is one staged tile: nc_box chunks x Rb rows.  Out-of-range boxes read zeros.
bool encode_plane(CUtensorMap* m, const uint16_t* plane, const Geom& g, const TcGeom& t) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !plane) return false;
    const cuuint64_t dims[3] = {8, (cuuint64_t)g.plane_pitch / 8, (cuuint64_t)g.plane_rows};
    const cuuint64_t strides[2] = {16, (cuuint64_t)g.plane_pitch * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)t.nc_box, (cuuint32_t)t.Rb};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(plane), dims, strides,
              box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Parts per tile for job g under class geometry t: a power of two up to
// cap, no larger than the fewest chunks of any of its tiles (the union of
// windows narrows at the left and right image edges), so that every part
// has at least one chunk of candidate columns.
int split_cap(const Geom& g, const TcGeom& t, int cap) {
    const int tiles_x = (g.n_rx + t.tx - 1) / t.tx;
    int min_chunks = 1 << 30;
    for (int bx = 0; bx < tiles_x; ++bx) {
        const int rx0 = bx * t.tx, rx_last = std::min(rx0 + t.tx - 1, g.n_rx - 1);
        const int X0 = std::max(0, rx0 * g.s - g.h), X1 = std::min(g.Wc - 1, rx_last * g.s + g.h);
        min_chunks = std::min(min_chunks, (X1 - X0 + 1 + t.kcols - 1) / t.kcols);
    }
    int w = 1;
    while (w * 2 <= cap && w * 2 <= min_chunks) w *= 2;
    return w;
}

bool make_job(TcJob& j, const Geom& g, const TcGeom& t, const TcArgs& a, int tile_begin) {
    j = TcJob{};
    if (!encode_plane(&j.map[0], a.plane0, g, t)) return false;
    if (t.f32 && !encode_plane(&j.map[1], a.plane1, g, t)) return false;
    j.plane[0] = a.plane0;
    j.plane[1] = a.plane1;
    j.pitch = g.plane_pitch;
    j.nsp = a.nsp;
    j.nrm = a.nrm;
    j.out_idx = a.out_idx;
    j.out_dist = a.out_dist;
    j.pool_idx = a.pool_idx;
    j.pool_score = a.pool_score;
    j.H = g.H; j.W = g.W; j.n_ry = g.n_ry; j.n_rx = g.n_rx; j.Hc = g.Hc; j.Wc = g.Wc;
    j.tiles_x = (g.n_rx + t.tx - 1) / t.tx;
    j.tile_begin = tile_begin;
    j.status = a.status;
    j.wsplit = 1;
    return true;
}

// Window-split merge: the parts' sorted lists of one reference merged into
// the first N entries by the lists' own order -- uint8: (distance, offset)
// ascending; float32 pool: (score descending, offset ascending) -- with
// empty entries (offset -1) last.  Every candidate is in exactly one part,
// so the result equals the list one pass over the whole window keeps.
struct MergeJob {
    const int32_t* idx;  // [wsplit][nR][N]
    const int32_t* val;  // distances (uint8) or score bits (float32), same layout
    int32_t* out_idx;    // [nR][N]
    int32_t* out_val;
    int nR, wsplit, ref_begin;
};
struct MergeParams {
    int N, f32, njobs, total;
    MergeJob jobs[kMaxJobs];
};

__global__ void __launch_bounds__(256) split_merge_kernel(const __grid_constant__ MergeParams P) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.total) return;
    int lo = 0, hi = P.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.jobs[mid].ref_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    const MergeJob& J = P.jobs[lo];
    const int r = t - J.ref_begin;
    int pos[4] = {0, 0, 0, 0};
    for (int i = 0; i < P.N; ++i) {
        int bq = 0;
        int32_t bid = 0, bv = 0;
        for (int q = 0; q < J.wsplit; ++q) {
            const int ps = pos[q] < P.N ? pos[q] : P.N - 1;
            const size_t e = ((size_t)q * J.nR + r) * P.N + ps;
            const int32_t id = pos[q] < P.N ? J.idx[e] : -1;
            const int32_t v = J.val[e];
            bool better;
            if (q == 0) better = true;
            else if (id < 0) better = false;
            else if (bid < 0) better = true;
            else if (P.f32) {
                const float a = __int_as_float(v), b = __int_as_float(bv);
                better = a > b || (a == b && id < bid);
            } else {
                better = v < bv || (v == bv && id < bid);
            }
            if (better) {
                bq = q;
                bid = id;
                bv = v;
            }
        }
        J.out_idx[(size_t)r * P.N + i] = bid;
        J.out_val[(size_t)r * P.N + i] = bv;
        ++pos[bq];
    }
}

cudaError_t launch_params(TcParams& P, cudaStream_t st) {
    const TcGeom& T = P.g;
    // at least 116 KB so that one CTA (one 512-column TMEM allocation) runs per SM
    const int smem = T.smem_total < 116 * 1024 ? 116 * 1024 : T.smem_total;
    void (*kern)(TcParams);
    int threads;
    if (T.nslots == 2) {
        threads = cta_threads(2);
        if (T.f32) kern = !T.tbits ? tc_match_kernel<32, true, 2, false>
                          : T.HL <= 24 ? tc_match_kernel<24, true, 2, true> : tc_match_kernel<32, true, 2, true>;
        else kern = T.HL <= 16 ? tc_match_kernel<16, false, 2, false> : tc_match_kernel<32, false, 2, false>;
    } else {
        threads = cta_threads(1);
        if (T.f32) kern = T.HL > 32 ? (T.tbits ? tc_match_kernel<0, true, 1, true> : tc_match_kernel<0, true, 1, false>)
                        : !T.tbits ? tc_match_kernel<32, true, 1, false>
                        : T.HL <= 24 ? tc_match_kernel<24, true, 1, true> : tc_match_kernel<32, true, 1, true>;
        else kern = T.HL <= 16 ? tc_match_kernel<16, false, 1, false>
                  : T.HL <= 32 ? tc_match_kernel<32, false, 1, false> : tc_match_kernel<0, false, 1, false>;
    }
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int per = T.nslots;
    int grid = (P.total_tiles + per - 1) / per;
    if (grid > num_sms()) grid = num_sms();
    if (grid < 1) grid = 1;
    kern<<<grid, threads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(const Geom& g) {
    TcGeom t{};
    return make_tc_geom(g, t);
}

// Tuner choices: every fitting tile configuration (make_tc_geom's
// candidates) times kSplitChoices window splits (1, 2 or 4 parts, bounded by
// the job's part-list room): choice = configuration * kSplitChoices + s.
int tc_num_choices(const Geom& g) {
    TcGeom t{};
    int n = 0;
    return make_tc_geom(g, t, -1, &n) ? n * kSplitChoices : 0;
}

bool tc_shape(const Geom& g, TcShape& s) {
    TcGeom t{};
    if (!make_tc_geom(g, t)) return false;
    s = TcShape{t.xs, t.ts, t.nslots, t.ty, t.tx, t.kcols, t.kbuf};
    return true;
}

int tc_column_parts(const Geom& g) {
    TcGeom t{};
    return make_tc_geom(g, t) ? t.xs : 1;
}

int tc_score_bits(const Geom& g) {
    TcGeom t{};
    return make_tc_geom(g, t) ? t.tbits : 0;
}

// Jobs that can share one persistent launch (same class geometry).
bool tc_same_class(const Geom& a, const Geom& b) {
    return a.dtype == b.dtype && a.Cp == b.Cp && a.p == b.p && a.h == b.h && a.s == b.s &&
           a.K == b.K && a.L == b.L && a.ncc == b.ncc;
}

cudaError_t launch_tc(const Geom& g, const TcArgs& a, cudaStream_t st) {
    return launch_tc_batch(&g, &a, 1, st);
}

cudaError_t launch_tc_batch(const Geom* gs, const TcArgs* as, int n, cudaStream_t st,
                            int* nlaunch, const int* choices) {
    int i = 0;
    if (nlaunch) *nlaunch = 0;
    while (i < n) {
        static thread_local TcParams P;
        P = TcParams{};
        const int choice = choices ? choices[i] : -1;
        // an explicit choice fixes the tile configuration and the split
        const int gchoice = choice >= 0 ? choice / kSplitChoices : -1;
        const int wsel = choice >= 0 ? 1 << (choice % kSplitChoices) : 0;  // 0: heuristic
        if (!make_tc_geom(gs[i], P.g, gchoice)) return cudaErrorNotSupported;
        P.fault = as[i].fault;
        P.inject = as[i].inject;
        int tiles = 0, nj = 0;
        const int first = i;
        while (i < n && nj < kMaxJobs && tc_same_class(gs[i], gs[i - nj]) &&
               (choices ? choices[i] : -1) == choice) {
            if (!make_job(P.jobs[nj], gs[i], P.g, as[i], tiles)) return cudaErrorInvalidValue;
            tiles += P.jobs[nj].tiles_x * ((gs[i].n_ry + P.g.ty - 1) / P.g.ty);
            ++nj;
            ++i;
        }
        // window split: by the heuristic only when the launch's tiles leave
        // SMs idle, then for every job that has part lists (wsplit of its
        // arguments); a tuned choice sets the parts itself
        const bool split = wsel > 0 || tiles < kSplitTarget;
        MergeParams M{};
        M.N = P.g.f32 ? P.g.HL : P.g.K;
        M.f32 = P.g.f32;
        tiles = 0;
        for (int j = 0; j < nj; ++j) {
            const TcArgs& a = as[first + j];
            TcJob& J = P.jobs[j];
            J.tile_begin = tiles;
            const int jt = J.tiles_x * ((J.n_ry + P.g.ty - 1) / P.g.ty);
            const int room = (a.split_idx && a.split_val) ? a.wsplit : 1;
            int w = split ? split_cap(gs[first + j], P.g, wsel > 0 ? std::min(wsel, room) : room) : 1;
            if (P.g.xs > 1) {  // column parts: always that many parts
                if (room < P.g.xs) return cudaErrorInvalidValue;
                w = P.g.xs;
            }
            if (w > 1) {
                J.wsplit = w;
                MergeJob& m = M.jobs[M.njobs++];
                m.nR = J.n_ry * J.n_rx;
                m.wsplit = w;
                m.ref_begin = M.total;
                m.idx = a.split_idx;
                m.val = a.split_val;
                M.total += m.nR;
                if (P.g.f32) {
                    m.out_idx = J.pool_idx;
                    m.out_val = reinterpret_cast<int32_t*>(J.pool_score);
                    J.pool_idx = a.split_idx;
                    J.pool_score = reinterpret_cast<float*>(a.split_val);
                } else {
                    m.out_idx = J.out_idx;
                    m.out_val = J.out_dist;
                    J.out_idx = a.split_idx;
                    J.out_dist = a.split_val;
                }
            }
            tiles += jt * J.wsplit;
        }
        P.njobs = nj;
        P.total_tiles = tiles;
        cudaError_t e = launch_params(P, st);
        if (e != cudaSuccess) return e;
        if (nlaunch) ++*nlaunch;
        if (M.njobs) {
            split_merge_kernel<<<(M.total + 255) / 256, 256, 0, st>>>(M);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (nlaunch) ++*nlaunch;
        }
    }
    return cudaSuccess;
}

int tc_window_split(const Geom& g) {
    TcGeom t{};
    if (!make_tc_geom(g, t)) return 1;
    if (t.xs > 1) return t.xs;
    const long long items = (long long)((g.n_rx + t.tx - 1) / t.tx) * ((g.n_ry + t.ty - 1) / t.ty);
    const long long want = kSplitTarget;
    int cap = 1;
    while (cap < kMaxSplit && items * cap < want) cap *= 2;
    return split_cap(g, t, cap);
}

}  // namespace bm
