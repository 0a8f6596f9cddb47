// selfconv_tc.cu -- (a3)-(a5): tcgen05 Self-Convolution cross term with the
// distance assembly and the per-reference top-K fused into the epilogue.
//
// What one CTA computes.  A tile of 128 reference patches (4 reference rows x
// 32 reference columns of the stride-s grid).  For every candidate j in the
// union of their search windows the tensor cores produce, per reference r,
//
//   v(r, j) = <X_r, X_j> - c * n_j          (n_j = ||X_j||^2, the box filter)
//
// i.e. the Self-Convolution C_r(j) of Eq. eq:selfConv (window-restricted as
// in the footnote to Eq. eq:unifySelfConv, summed over channels as S(.) in
// Eq. equ:self-convMM) minus the norm term, which is Theorem 1's
// b = vec(C_r) - 0.5 h_X (.) h_X: the K largest entries of b are the K
// nearest candidates, and d = ||X_r||^2 - 2 b (Lemma 2).  The norm term is an
// extra K-step of the same MMA (A = constant coefficients, B = n_j split into
// three bf16 pieces), so TMEM already holds the score.
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
// Operand layout (no im2col in HBM).  A (references) is K-major in the
// canonical no-swizzle core-matrix layout, staged once per CTA.  B
// (candidates) is formed in shared memory per chunk of candidate columns as
// "column strips": for candidate column j and 16-byte chunk q of a patch row,
// strip[q][j][row] holds the 8 elements starting at pixel (X0 + j) of image
// row (Y0 + row).  Candidate n = j * Rb + row (column-major) then reads patch
// row u at strip[q][j][row + u]: eight consecutive candidates are eight
// consecutive 16-byte rows -- exactly a no-swizzle K-major core matrix -- so
// every K-step is a plain descriptor with SBO = 128 B and LBO = 16 B (next
// patch row) or the q-strip pitch (next chunk of the same row).
//
// Warp roles: warps 0..EW-1 epilogue (warp w reads TMEM lanes 32(w%4)..+31;
// with EW = 8 two warps share each lane quarter and take alternate candidate
// columns, each keeping its own list, merged at the end of the tile), the
// next three warps producers (strip formation from the bf16 planes), the last
// warp TMEM allocation + single-thread MMA issue.
// Pipelines: kStages shared-memory stages (mbarriers full/empty) and two
// 256-column TMEM accumulators (tfull/tempty).  Every wait is bounded; on
// timeout the CTA sets *status, drains and frees its TMEM.
#include "bm_internal.h"

#include <cuda_bf16.h>

namespace bm {
namespace {

constexpr int kProducers = 96;  // three producer warps
// Threads of a CTA with EW epilogue warps: EW + 3 producer warps + 1 MMA warp.
template <int EW>
__host__ __device__ constexpr int cta_threads() { return EW * 32 + kProducers + 32; }
constexpr int kStages = 3;
constexpr int kTmemCols = 512;
constexpr int kBufCols = 256;
constexpr float kEps = 6.103515625e-05f;  // 2^-14
constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kSmemLimit = 227 * 1024;
constexpr int kBuf = 32;   // per-lane append buffer (entries) between merges
constexpr int kBatch = 8;  // keys merged into the register list at a time

// Class-wide geometry of one launch (every job shares patch, window, stride,
// K, channel padding and dtype; image sizes are per job).
struct TcGeom {
    int Cp, p, h, s, K, HL;
    int rr, rc, wgx, ty, tx;  // lane -> reference mapping and tile shape (references)
    int pw, p_eff, nkc, Rb, kcols;
    int nslots, bufcols;      // tiles in flight per CTA, TMEM columns per accumulator
    int qpitch, plane_stage, ns_bytes, stage_bytes;
    int f32;
    int off_a, a_bytes, off_an, off_stage, off_heap, off_buf, off_bar, smem_total;
};

// One image of a launch.
struct TcJob {
    const uint16_t* plane0;
    const uint16_t* plane1;
    const void* nrm;
    int32_t* out_idx;     // uint8: final indices
    int32_t* out_dist;    // uint8: final distances
    int32_t* pool_idx;    // float32: pool
    float* pool_score;
    int H, W, n_ry, n_rx, Hc, Wc, plane_pitch;
    int tiles_x, tile_begin;  // tiles along x; index of the job's first tile
};

constexpr int kMaxJobs = 160;  // jobs per launch (kept inline in the kernel parameters)

struct TcParams {
    TcGeom g;
    int njobs, total_tiles;
    int* status;
    TcJob jobs[kMaxJobs];
};

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
template <>
__device__ __forceinline__ void tmem_ld_blocks<2>(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + 0u), "r"(taddr + 16u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld_blocks<4>(uint32_t taddr, float* v) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%65];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%66];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%67];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr + 0u), "r"(taddr + 16u), "r"(taddr + 32u), "r"(taddr + 48u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float max3(float a, float b, float c) {
    float m;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    return m;
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
// x = hi + mid + lo exactly for any float with <= 24 significant bits.
__device__ __forceinline__ void split3(float x, uint16_t& hi, uint16_t& mid, uint16_t& lo) {
    hi = bf16_bits(x);
    float r1 = x - bf16_val(hi);
    mid = bf16_bits(r1);
    float r2 = r1 - bf16_val(mid);
    lo = bf16_bits(r2);
}

__device__ __forceinline__ unsigned orderable(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_orderable(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// 16 bytes of a bf16 plane row starting at element e0 (any alignment).
__device__ __forceinline__ uint4 load_shifted16(const uint16_t* row, int e0) {
    const int a0 = e0 & ~7, sh = e0 & 7;
    const uint4 A = __ldg(reinterpret_cast<const uint4*>(row + a0));
    if (sh == 0) return A;
    const uint4 B = __ldg(reinterpret_cast<const uint4*>(row + a0 + 8));
    const uint32_t w[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
    const int j = sh >> 1;
    uint32_t s[5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
        s[i] = j == 0 ? w[i] : j == 1 ? w[i + 1] : j == 2 ? w[i + 2] : w[i + 3];
    const uint32_t f = (sh & 1) * 16;
    uint4 o;
    o.x = __funnelshift_r(s[0], s[1], f);
    o.y = __funnelshift_r(s[1], s[2], f);
    o.z = __funnelshift_r(s[2], s[3], f);
    o.w = __funnelshift_r(s[3], s[4], f);
    return o;
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

// Compare-exchange: x <- min, y <- max.
__device__ __forceinline__ void cmpx(unsigned long long& x, unsigned long long& y) {
    const bool s = y < x;
    const unsigned long long lo = s ? y : x, hi = s ? x : y;
    x = lo;
    y = hi;
}
// Bitonic sort of N registers, ascending.
template <int N>
__device__ __forceinline__ void bitonic_sort(unsigned long long (&v)[N]) {
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
template <int N>
__device__ __forceinline__ void bitonic_merge(unsigned long long (&v)[N]) {
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
// than a full insertion pass per key.  Entries 0..cap-1 are the
// answer (cap <= LC); extra entries only make the list a superset.
template <int LC>
struct RegTopK {
    unsigned long long a[LC];
    int cap;
    __device__ __forceinline__ void init(int c) {
        cap = c;
#pragma unroll
        for (int i = 0; i < LC; ++i) a[i] = kEmpty;
    }
    __device__ __forceinline__ void merge_batch(unsigned long long (&b)[kBatch]) {
        bitonic_sort<kBatch>(b);
#pragma unroll
        for (int i = 0; i < LC; ++i) {
            const int bi = LC - 1 - i;
            if (bi < kBatch) a[i] = b[bi] < a[i] ? b[bi] : a[i];
        }
        bitonic_merge<LC>(a);
    }
    __device__ __forceinline__ unsigned long long kth() const {  // entry cap-1
        unsigned long long r = 0;
#pragma unroll
        for (int i = 0; i < LC; ++i) {
            const unsigned long long x = i < cap ? a[i] : 0ull;
            r = x > r ? x : r;
        }
        return r;
    }
};

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
    if constexpr (LC > 0) t = reg.kth();
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
};

// Tile t of the launch: its job (binary search over the jobs' first tiles)
// and the union of its references' clipped windows.
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
    const int lt = t - J.tile_begin;
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
    return T;
}

// Tile of slot k's g-th turn in CTA b (static round robin over the launch).
__device__ __forceinline__ int slot_tile(int b, int g, int k, int nslots, int grid) {
    return b + (g * nslots + k) * grid;
}

// ---------------------------------------------------------------- the kernel
//
// Persistent: CTA b walks the tiles b, b + G, b + 2G, ... of every job of
// the launch, NS tiles in flight ("slots").  Slot k owns epilogue warps
// 4k..4k+3, its own A operand region and two TMEM accumulators; the
// producers and the MMA thread alternate between the slots' chunks, so the
// epilogue of one tile overlaps the MMAs of the other.
template <int LC, bool F32, int NS>
__global__ void __launch_bounds__(cta_threads<4 * NS>(), 1)
tc_match_kernel(const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcGeom& G = P.g;
    constexpr bool kF32 = F32;
    constexpr int EW = 4 * NS;
    constexpr int kThreads = cta_threads<EW>();
    constexpr int kMmaWarp = EW + 3;
    constexpr int kEpi = EW * 32;  // epilogue threads (pending-buffer stride)
    constexpr int nplanes = kF32 ? 2 : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grid = gridDim.x, cta = blockIdx.x;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G.off_bar);
    // barrier slots: full[kStages], empty[kStages], tfull[NS][2], tempty[NS][2],
    // afull[NS], aempty[NS], done
    const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + kStages);
    const uint32_t bar_tfull = smem_u32(bars + 2 * kStages);
    const uint32_t bar_tempty = smem_u32(bars + 2 * kStages + 2 * NS);
    const uint32_t bar_afull = smem_u32(bars + 2 * kStages + 4 * NS);
    const uint32_t bar_aempty = smem_u32(bars + 2 * kStages + 5 * NS);
    const uint32_t bar_done = smem_u32(bars + 2 * kStages + 6 * NS);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 6 * NS + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(bar_full + 8 * i, kProducers);
            mbar_init(bar_empty + 8 * i, 1);
        }
        for (int i = 0; i < 2 * NS; ++i) {
            mbar_init(bar_tfull + 8 * i, 1);
            mbar_init(bar_tempty + 8 * i, 128);
        }
        for (int k = 0; k < NS; ++k) {
            mbar_init(bar_afull + 8 * k, kProducers);
            mbar_init(bar_aempty + 8 * k, 1);
        }
        mbar_init(bar_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
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
    // stage buffers start zeroed so padding rows are finite
    for (int t = threadIdx.x; t < kStages * G.stage_bytes / 16; t += kThreads)
        reinterpret_cast<uint4*>(smem + G.off_stage)[t] = make_uint4(0, 0, 0, 0);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp >= EW && warp < kMmaWarp) {
        // ------------------------------------------------------------ producers
        const int pt = threadIdx.x - kEpi;
        const int strip_items = nplanes * G.pw * G.kcols * G.Rb;
        const int norm_items = G.kcols * G.Rb;
        TileInfo ti[NS];
        int chunk[NS], turn[NS];
        bool active[NS];
        for (int k = 0; k < NS; ++k) {
            turn[k] = 0;
            chunk[k] = 0;
            const int t = slot_tile(cta, 0, k, NS, grid);
            active[k] = t < P.total_tiles;
            if (active[k]) ti[k] = tile_info(P, t);
        }
        int step = 0, next = 0;
        bool ok = true;
        while (ok) {
            int k = next;
            if (!active[k]) k = NS - 1 - k;
            if (!active[k]) break;
            next = NS - 1 - k;
            const TileInfo& T = ti[k];
            const TcJob& J = *T.job;
            if (chunk[k] == 0) {
                // new tile for slot k: stage its A operand once the previous
                // tile's MMAs are done with the region
                if (turn[k] > 0 && !mbar_wait(bar_aempty + 8 * k, (turn[k] - 1) & 1, abort_flag, 5)) {
                    ok = false;
                    break;
                }
                const int items = 128 * G.nkc * nplanes;
                for (int t0 = pt; t0 < items; t0 += 4 * kProducers) {
                    uint4 val[4];
                    int dst[4];
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4) {
                        const int t = t0 + u4 * kProducers;
                        dst[u4] = -1;
                        val[u4] = make_uint4(0, 0, 0, 0);
                        if (t >= items) continue;
                        const int pl = t / (128 * G.nkc), it = t % (128 * G.nkc);
                        const int m = it / G.nkc, kc = it % G.nkc;
                        const int u = kc / G.pw, q = kc % G.pw;
                        const int mw = m >> 5, ml = m & 31;
                        const int ry = T.ry0 + (mw / G.wgx) * G.rr + ml / G.rc;
                        const int rx = T.rx0 + (mw % G.wgx) * G.rc + ml % G.rc;
                        dst[u4] = k * G.a_bytes * nplanes + pl * G.a_bytes +
                                  (m >> 3) * G.nkc * 128 + kc * 128 + (m & 7) * 16;
                        if (ry < J.n_ry && rx < J.n_rx && u < G.p) {
                            const uint16_t* plane = pl ? J.plane1 : J.plane0;
                            const uint16_t* row = plane + (size_t)(ry * G.s + u) * J.plane_pitch;
                            uint4 v = load_shifted16(row, rx * G.s * G.Cp + 8 * q);
                            // zero the elements beyond the patch row (p * Cp elements)
                            const int valid = G.p * G.Cp - 8 * q;
                            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                if (2 * i >= valid) w[i] = 0;
                                else if (2 * i + 1 >= valid) w[i] &= 0xffffu;
                                if (!kF32) {
                                    // uint8: A = 2 (x - 128), exact in bf16: MMA gives 2 <X_r, X_j>
                                    const float lo_f = 2.0f * bf16_val((uint16_t)(w[i] & 0xffffu));
                                    const float hi_f = 2.0f * bf16_val((uint16_t)(w[i] >> 16));
                                    w[i] = (uint32_t)bf16_bits(lo_f) | ((uint32_t)bf16_bits(hi_f) << 16);
                                }
                            }
                            val[u4] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4)
                        if (dst[u4] >= 0)
                            *reinterpret_cast<uint4*>(smem + G.off_a + dst[u4]) = val[u4];
                }
                fence_proxy_async();
                mbar_arrive(bar_afull + 8 * k);
            }
            // one chunk of candidate columns of slot k's tile
            const int stage = step % kStages, use = step / kStages;
            if (use > 0 && !mbar_wait(bar_empty + 8 * stage, (use - 1) & 1, abort_flag, 1)) break;
            uint8_t* sb = smem + G.off_stage + stage * G.stage_bytes;
            const int jc0 = chunk_order(chunk[k], T.nchunks, T.center_chunk) * G.kcols;
            const int kc_here = min(G.kcols, T.NX - jc0);
            for (int t0 = pt; t0 < strip_items; t0 += 4 * kProducers) {
                uint4 val[4];
                int dst[4];
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4) {
                    const int t = t0 + u4 * kProducers;
                    dst[u4] = -1;
                    val[u4] = make_uint4(0, 0, 0, 0);
                    if (t >= strip_items) continue;
                    int r = t;
                    const int row = r % G.Rb; r /= G.Rb;
                    const int jl = r % G.kcols; r /= G.kcols;
                    const int q = r % G.pw;
                    const int pl = r / G.pw;
                    if (jl >= kc_here) continue;
                    dst[u4] = pl * G.plane_stage + q * G.qpitch + (jl * G.Rb + row) * 16;
                    if (row < T.NR + G.p_eff - 1) {  // rows past that feed no real candidate
                        const uint16_t* plane = pl ? J.plane1 : J.plane0;
                        const uint16_t* prow = plane + (size_t)(T.Y0 + row) * J.plane_pitch;
                        val[u4] = load_shifted16(prow, (T.X0 + jc0 + jl) * G.Cp + 8 * q);
                    }
                }
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4)
                    if (dst[u4] >= 0) *reinterpret_cast<uint4*>(sb + dst[u4]) = val[u4];
            }
            uint8_t* nsb = sb + nplanes * G.plane_stage;
            const int* nrm_i = static_cast<const int*>(J.nrm);
            const float* nrm_f = static_cast<const float*>(J.nrm);
            for (int t = pt; t < norm_items; t += kProducers) {
                const int row = t % G.Rb, jl = t / G.Rb;
                if (jl >= kc_here) continue;
                uint16_t hi = 0, mid = 0, lo = 0;
                if (row < T.NR) {
                    const size_t ni = (size_t)(T.Y0 + row) * J.Wc + (T.X0 + jc0 + jl);
                    const float w = kF32 ? nrm_f[ni] : (float)nrm_i[ni];
                    split3(w, hi, mid, lo);
                } else {
                    hi = bf16_bits(1.0e18f);  // no real candidate: never selected
                }
                uint4 val;
                if (kF32) {
                    val = make_uint4(hi | (uint32_t(mid) << 16), lo | (uint32_t(hi) << 16),
                                     mid | (uint32_t(lo) << 16), 0u);
                } else {
                    val = make_uint4(hi | (uint32_t(mid) << 16), lo, 0u, 0u);
                }
                *reinterpret_cast<uint4*>(nsb + (jl * G.Rb + row) * 16) = val;
            }
            fence_proxy_async();
            mbar_arrive(bar_full + 8 * stage);
            ++step;
            if (++chunk[k] == T.nchunks) {
                chunk[k] = 0;
                ++turn[k];
                const int t = slot_tile(cta, turn[k], k, NS, grid);
                active[k] = t < P.total_tiles;
                if (active[k]) ti[k] = tile_info(P, t);
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t an = smem_u32(smem + G.off_an);
            const uint32_t sbo_a = G.nkc * 128;
            const uint32_t lbo_b = G.pw == 1 ? 16u : (uint32_t)G.qpitch;
            int nchunks[NS], center[NS], NX[NS], chunk[NS], turn[NS], q[NS];
            bool active[NS];
            for (int k = 0; k < NS; ++k) {
                chunk[k] = turn[k] = q[k] = 0;
                const int t = slot_tile(cta, 0, k, NS, grid);
                active[k] = t < P.total_tiles;
                if (active[k]) {
                    const TileInfo T = tile_info(P, t);
                    nchunks[k] = T.nchunks; center[k] = T.center_chunk; NX[k] = T.NX;
                }
            }
            int step = 0, next = 0;
            while (true) {
                int k = next;
                if (!active[k]) k = NS - 1 - k;
                if (!active[k]) break;
                next = NS - 1 - k;
                if (chunk[k] == 0 &&
                    !mbar_wait(bar_afull + 8 * k, turn[k] & 1, abort_flag, 6))
                    break;
                const int buf = q[k] & 1, ub = q[k] >> 1;
                if (ub > 0 &&
                    !mbar_wait(bar_tempty + 8 * (2 * k + buf), (ub - 1) & 1, abort_flag, 2))
                    break;
                const int stage = step % kStages, use = step / kStages;
                if (!mbar_wait(bar_full + 8 * stage, use & 1, abort_flag, 3)) break;
                tc_fence_after();
                const int jc0 = chunk_order(chunk[k], nchunks[k], center[k]) * G.kcols;
                const int kc_here = min(G.kcols, NX[k] - jc0);
                const uint32_t idesc = idesc_bf16(128, kc_here * G.Rb);
                const uint32_t d = tmem_base + (2 * k + buf) * G.bufcols;
                const uint32_t sb = smem_u32(smem + G.off_stage + stage * G.stage_bytes);
                const uint32_t a0 = smem_u32(smem + G.off_a + k * G.a_bytes * nplanes);
                const uint32_t a1 = a0 + G.a_bytes;
                uint32_t acc = 0;
                for (int t = 0; t < G.nkc / 2; ++t) {
                    const int kc = 2 * t;
                    const int u = kc / G.pw, qq = kc % G.pw;
                    const uint32_t boff = qq * G.qpitch + u * 16;
                    const uint64_t da0 = sdesc(a0 + kc * 128, 128, sbo_a);
                    const uint64_t db0 = sdesc(sb + boff, lbo_b, 128);
                    mma_bf16(d, da0, db0, idesc, acc);
                    acc = 1;
                    if (kF32) {
                        const uint64_t db1 = sdesc(sb + G.plane_stage + boff, lbo_b, 128);
                        const uint64_t da1 = sdesc(a1 + kc * 128, 128, sbo_a);
                        mma_bf16(d, da0, db1, idesc, 1);
                        mma_bf16(d, da1, db0, idesc, 1);
                    }
                }
                const uint32_t nsb = sb + nplanes * G.plane_stage;
                mma_bf16(d, sdesc(an, 128, 256), sdesc(nsb, 16, 128), idesc, 1);
                mma_commit(bar_empty + 8 * stage);
                mma_commit(bar_tfull + 8 * (2 * k + buf));
                ++step;
                ++q[k];
                if (++chunk[k] == nchunks[k]) {
                    mma_commit(bar_aempty + 8 * k);  // A region of slot k free once these finish
                    chunk[k] = 0;
                    ++turn[k];
                    const int t = slot_tile(cta, turn[k], k, NS, grid);
                    active[k] = t < P.total_tiles;
                    if (active[k]) {
                        const TileInfo T = tile_info(P, t);
                        nchunks[k] = T.nchunks; center[k] = T.center_chunk; NX[k] = T.NX;
                    }
                }
            }
            // drain: wait for every MMA issued by this thread before TMEM is freed
            mma_commit(bar_done);
            const unsigned long long t0 = globaltimer();
            while (!mbar_try_wait(bar_done, 0) && globaltimer() - t0 < kWaitNs) {
            }
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
        unsigned long long* pend =
            reinterpret_cast<unsigned long long*>(smem + G.off_buf) + threadIdx.x;
        Heap heap{reinterpret_cast<unsigned long long*>(smem + G.off_heap) + (threadIdx.x & 127), G.HL};
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        int qc = 0;  // slot-local chunk counter (TMEM buffer phase)
        for (int turn = 0; !*abort_flag; ++turn) {
            const int tile = slot_tile(cta, turn, k, NS, grid);
            if (tile >= P.total_tiles) break;
            const TileInfo T = tile_info(P, tile);
            const TcJob& J = *T.job;
            RegTopK<LC == 0 ? 1 : LC> reg;
            reg.init(G.HL);
            if constexpr (LC == 0) {
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
            float thr = -__int_as_float(0x7f800000);  // -inf while the list has empty slots
            int cnt = 0;
            for (int c = 0; c < T.nchunks; ++c, ++qc) {
                const int buf = qc & 1, ub = qc >> 1;
                if (!mbar_wait(bar_tfull + 8 * (2 * k + buf), ub & 1, abort_flag, 4)) break;
                tc_fence_after();
                const int jc0 = chunk_order(c, T.nchunks, T.center_chunk) * G.kcols;
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
                    for (int bb = 0; bb < nblk; ++bb) {
                        float w[16];
                        tmem_ld_blocks<1>(colbase + 16 * bb, w);
                        const int b = b0 + bb;
                        // this lane's valid rows of block b: [i0, i1] (may be empty)
                        const int i0 = lo - 16 * b, i1 = xok ? hi - 16 * b : -1;
                        const float ninf = -__int_as_float(0x7f800000);
                        float m = ninf;
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const float a = (i >= i0 && i <= i1) ? w[i] : ninf;
                            const float c2 = (i + 1 >= i0 && i + 1 <= i1) ? w[i + 1] : ninf;
                            m = max3(m, a, c2);
                        }
                        const bool hit = m >= thr;
                        if (!__any_sync(0xffffffffu, hit)) continue;  // next block
                        if (hit) {
                            const int ybase = T.Y0 + 16 * b;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                if (i >= i0 && i <= i1 && w[i] >= thr) {
                                    pend[cnt * kEpi] =
                                        ((unsigned long long)__float_as_uint(w[i]) << 32) |
                                        (unsigned)((ybase + i) * J.W + xc);
                                    ++cnt;
                                }
                            }
                        }
                        // keep room for the next block's appends
                        if (__any_sync(0xffffffffu, cnt > kBuf - 16))
                            merge_pending<LC, kF32, kEpi>(G, nrm_i, nr_i, pend, cnt, thr, reg, heap);
                    }
                }
                tc_fence_before();
                mbar_arrive(bar_tempty + 8 * (2 * k + buf));
            }
            if (__any_sync(0xffffffffu, cnt > 0))
                reg = final_merge<LC, kF32, kEpi>(G, nrm_i, nr_i, pend, cnt, reg, heap.h);
            // ---- write results
            if (lane_ok && !*abort_flag) {
                const size_t ref = (size_t)ry * J.n_rx + rx;
                if constexpr (LC == 0 && !kF32) heap.sort();
                const int nout = kF32 ? G.HL : G.K;
                auto emit = [&](int i, unsigned long long key) {
                    if (kF32) {
                        // pool: any order; the re-rank kernel ranks it
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
                if constexpr (LC > 0) {
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
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(P.status, 0x100 + *abort_flag);
}

// Class geometry for a job shape: lane mapping, strips, slots, shared memory.
bool make_tc_geom(const Geom& g, TcGeom& t) {
    t.Cp = g.Cp; t.p = g.p; t.h = g.h; t.s = g.s; t.K = g.K;
    t.pw = g.pw; t.p_eff = g.p_eff; t.nkc = g.p_eff * g.pw;
    t.f32 = g.dtype == kF32;
    t.HL = t.f32 ? g.L : g.K;
    // two tiles in flight when the list lives in registers and a strip fits
    // a 128-column accumulator; one otherwise
    for (int ns = 2; ns >= 1; --ns) {
        if (ns == 2 && t.HL > 32) continue;
        const int bufcols = kTmemCols / (2 * ns);
        // lane -> reference mapping: rr reference rows x rc columns per warp,
        // a wgy x wgx grid of 4 warps; least MMA work (union columns x strip
        // rows), ties to the earlier (narrower) entry
        static const int kMaps[6][2] = {{8, 2}, {16, 4}, {32, 4}, {8, 4}, {4, 4}, {1, 1}};
        long long best = -1;
        for (const auto& mp : kMaps) {
            const int rr = mp[0], wgx = mp[1], rc = 32 / rr, wgy = 4 / wgx;
            const int ty = wgy * rr, tx = wgx * rc;
            const int nr_max = (ty - 1) * g.s + 2 * g.h + 1;
            const int nx_max = (tx - 1) * g.s + 2 * g.h + 1;
            const int rb = (nr_max + g.p_eff - 1 + 15) / 16 * 16;
            if (rb > bufcols) continue;
            const long long work = (long long)nx_max * rb;
            if (best < 0 || work < best) {
                best = work;
                t.rr = rr; t.rc = rc; t.wgx = wgx; t.ty = ty; t.tx = tx; t.Rb = rb;
            }
        }
        if (best < 0) continue;
        t.nslots = ns;
        t.bufcols = bufcols;
        break;
    }
    if (t.Rb <= 0 || t.Rb > kBufCols) return false;
    t.kcols = t.bufcols / t.Rb;
    const int strip_rows = t.kcols * t.Rb + g.p_eff + 16;
    t.qpitch = strip_rows * 16;
    t.plane_stage = t.pw * t.qpitch;
    t.ns_bytes = (t.kcols * t.Rb + 16) * 16;
    const int nplanes = t.f32 ? 2 : 1;
    t.stage_bytes = (nplanes * t.plane_stage + t.ns_bytes + 127) / 128 * 128;
    int off = 0;
    t.a_bytes = 128 * t.nkc * 16;
    t.off_a = off; off += t.nslots * nplanes * t.a_bytes;
    t.off_an = off; off += 128 * 2 * 16;
    t.off_stage = off; off += kStages * t.stage_bytes;
    t.off_heap = off; off += t.HL > 32 ? 128 * t.HL * 8 : 0;
    t.off_buf = off; off += 4 * t.nslots * 32 * kBuf * 8;
    t.off_bar = off; off += (2 * kStages + 6 * t.nslots + 1) * 8 + 16;
    t.smem_total = (off + 1023) / 1024 * 1024;
    return t.smem_total <= kSmemLimit;
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

TcJob make_job(const Geom& g, const TcGeom& t, const TcArgs& a, int tile_begin) {
    TcJob j{};
    j.plane0 = a.plane0;
    j.plane1 = a.plane1;
    j.nrm = a.nrm;
    j.out_idx = a.out_idx;
    j.out_dist = a.out_dist;
    j.pool_idx = a.pool_idx;
    j.pool_score = a.pool_score;
    j.H = g.H; j.W = g.W; j.n_ry = g.n_ry; j.n_rx = g.n_rx; j.Hc = g.Hc; j.Wc = g.Wc;
    j.plane_pitch = g.plane_pitch;
    j.tiles_x = (g.n_rx + t.tx - 1) / t.tx;
    j.tile_begin = tile_begin;
    return j;
}

cudaError_t launch_params(TcParams& P, cudaStream_t st) {
    const TcGeom& T = P.g;
    const int smem = T.smem_total < 116 * 1024 ? 116 * 1024 : T.smem_total;
    void (*kern)(TcParams);
    int threads;
    if (T.nslots == 2) {
        threads = cta_threads<8>();
        if (T.f32) kern = tc_match_kernel<32, true, 2>;
        else kern = T.HL <= 16 ? tc_match_kernel<16, false, 2> : tc_match_kernel<32, false, 2>;
    } else {
        threads = cta_threads<4>();
        if (T.f32) kern = T.HL <= 32 ? tc_match_kernel<32, true, 1> : tc_match_kernel<0, true, 1>;
        else kern = T.HL <= 16 ? tc_match_kernel<16, false, 1>
                  : T.HL <= 32 ? tc_match_kernel<32, false, 1> : tc_match_kernel<0, false, 1>;
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

// Jobs that can share one persistent launch (same class geometry).
bool tc_same_class(const Geom& a, const Geom& b) {
    return a.dtype == b.dtype && a.Cp == b.Cp && a.p == b.p && a.h == b.h && a.s == b.s &&
           a.K == b.K && a.L == b.L;
}

cudaError_t launch_tc(const Geom& g, const TcArgs& a, cudaStream_t st) {
    return launch_tc_batch(&g, &a, 1, st);
}

cudaError_t launch_tc_batch(const Geom* gs, const TcArgs* as, int n, cudaStream_t st) {
    int i = 0;
    while (i < n) {
        static thread_local TcParams P;
        P = TcParams{};
        if (!make_tc_geom(gs[i], P.g)) return cudaErrorNotSupported;
        P.status = as[i].status;
        int tiles = 0, nj = 0;
        while (i < n && nj < kMaxJobs && tc_same_class(gs[i], gs[i - nj])) {
            P.jobs[nj] = make_job(gs[i], P.g, as[i], tiles);
            tiles += P.jobs[nj].tiles_x * ((gs[i].n_ry + P.g.ty - 1) / P.g.ty);
            ++nj;
            ++i;
        }
        P.njobs = nj;
        P.total_tiles = tiles;
        cudaError_t e = launch_params(P, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bm
