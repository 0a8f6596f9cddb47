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
//   uint8 : bf16 operands are exact (0..255), products and all partial sums
//           are integers below 2^24, so the FP32 accumulation is exact; the
//           norm term is floor(n_j / 2) with coefficient -1 and the parity of
//           n_j is restored in the exact key d = n_r - 2 v + (n_j & 1).
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
// Warp roles (288 threads): warps 0-3 epilogue (TMEM lanes 32w..32w+31 =
// reference row w of the tile), warps 4-7 producers (strip formation from
// the bf16 planes), warp 8 TMEM allocation + single-thread MMA issue.
// Pipelines: kStages shared-memory stages (mbarriers full/empty) and two
// 256-column TMEM accumulators (tfull/tempty).  Every wait is bounded; on
// timeout the CTA sets *status, drains and frees its TMEM.
#include "bm_internal.h"

#include <cuda_bf16.h>

namespace bm {
namespace {

constexpr int kThreads = 288;
constexpr int kMmaWarp = 8;
constexpr int kStages = 3;
constexpr int kTmemCols = 512;
constexpr int kBufCols = 256;
constexpr float kEps = 6.103515625e-05f;  // 2^-14
constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kSmemLimit = 227 * 1024;

struct TcGeom {
    int H, W, Cp, p, h, s, K, HL, n_ry, n_rx, Hc, Wc;
    int pw, p_eff, nkc, Rb, kcols;
    int qpitch, plane_stage, ns_bytes, stage_bytes;
    int plane_pitch;
    int f32;
    int off_a0, off_a1, off_an, off_stage, off_heap, off_bar, smem_total;
};

struct TcParams {
    TcGeom g;
    const uint16_t* plane0;
    const uint16_t* plane1;
    const void* nrm;
    int32_t* out_idx;
    int32_t* out_dist;
    int32_t* pool_idx;
    float* pool_score;
    int* status;
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
// Bounded wait on one mbarrier phase.  False on timeout or abort.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
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
// 32 lanes x 16 consecutive columns, waited before returning.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
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

// Max-heap of u64 keys per epilogue thread, element i at h[i * 128].
struct Heap {
    unsigned long long* h;
    int n;
    __device__ __forceinline__ unsigned long long top() const { return h[0]; }
    __device__ void replace_top(unsigned long long key) {
        int i = 0;
        while (true) {
            int l = 2 * i + 1;
            if (l >= n) break;
            int r = l + 1;
            unsigned long long cv = h[l * 128];
            int c = l;
            if (r < n) {
                unsigned long long rv = h[r * 128];
                if (rv > cv) { cv = rv; c = r; }
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

// ---------------------------------------------------------------- the kernel
__global__ void __launch_bounds__(kThreads, 1) tc_match_kernel(const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcGeom& G = P.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int ry0 = blockIdx.y * 4, rx0 = blockIdx.x * 32;
    const int ry_last = min(ry0 + 3, G.n_ry - 1), rx_last = min(rx0 + 31, G.n_rx - 1);
    const int Y0 = max(0, ry0 * G.s - G.h), Y1 = min(G.Hc - 1, ry_last * G.s + G.h);
    const int X0 = max(0, rx0 * G.s - G.h), X1 = min(G.Wc - 1, rx_last * G.s + G.h);
    const int NR = Y1 - Y0 + 1, NX = X1 - X0 + 1;
    const int nchunks = (NX + G.kcols - 1) / G.kcols;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G.off_bar);
    const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + kStages);
    const uint32_t bar_tfull = smem_u32(bars + 2 * kStages);
    const uint32_t bar_tempty = smem_u32(bars + 2 * kStages + 2);
    const uint32_t bar_done = smem_u32(bars + 2 * kStages + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(bar_full + 8 * i, 128);
            mbar_init(bar_empty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar_tfull + 8 * i, 1);
            mbar_init(bar_tempty + 8 * i, 128);
        }
        mbar_init(bar_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), kTmemCols);

    // ---- A: reference patches, K-major core matrices [group][kchunk][8 rows x 16 B]
    {
        const int nplanes = G.f32 ? 2 : 1;
        const int items = 128 * G.nkc;
        for (int t = threadIdx.x; t < items * nplanes; t += kThreads) {
            const int pl = t / items, it = t % items;
            const int m = it / G.nkc, kc = it % G.nkc;
            const int u = kc / G.pw, q = kc % G.pw;
            const int ry = ry0 + (m >> 5), rx = rx0 + (m & 31);
            uint4 val = make_uint4(0, 0, 0, 0);
            if (ry < G.n_ry && rx < G.n_rx && u < G.p) {
                const uint16_t* plane = pl ? P.plane1 : P.plane0;
                const uint16_t* row = plane + (size_t)(ry * G.s + u) * G.plane_pitch;
                val = load_shifted16(row, rx * G.s * G.Cp + 8 * q);
                // zero the elements beyond the patch row (p * Cp elements)
                const int valid = G.p * G.Cp - 8 * q;
                if (valid < 8) {
                    uint32_t w[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (2 * i >= valid) w[i] = 0;
                        else if (2 * i + 1 >= valid) w[i] &= 0xffffu;
                    }
                    val = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            uint8_t* base = smem + (pl ? G.off_a1 : G.off_a0);
            *reinterpret_cast<uint4*>(base + (size_t)(m >> 3) * G.nkc * 128 + kc * 128 +
                                      (m & 7) * 16) = val;
        }
        // A_norm: [group][2 kchunks][8 x 16 B]; row = coefficients of the norm pieces
        for (int t = threadIdx.x; t < 128 * 2; t += kThreads) {
            const int m = t >> 1, kc = t & 1;
            uint16_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (kc == 0) {
                const uint16_t cn = bf16_bits(G.f32 ? -0.5f : -1.0f);
                c[0] = c[1] = c[2] = cn;
                if (G.f32) c[3] = c[4] = c[5] = bf16_bits(kEps);
            }
            uint4 val = make_uint4(c[0] | (uint32_t(c[1]) << 16), c[2] | (uint32_t(c[3]) << 16),
                                   c[4] | (uint32_t(c[5]) << 16), c[6] | (uint32_t(c[7]) << 16));
            *reinterpret_cast<uint4*>(smem + G.off_an + (m >> 3) * 256 + kc * 128 + (m & 7) * 16) = val;
        }
    }
    // stage buffers start zeroed so padding rows are finite
    for (int t = threadIdx.x; t < kStages * G.stage_bytes / 16; t += kThreads)
        reinterpret_cast<uint4*>(smem + G.off_stage)[t] = make_uint4(0, 0, 0, 0);
    // epilogue threads: empty heaps
    if (threadIdx.x < 128) {
        unsigned long long* h = reinterpret_cast<unsigned long long*>(smem + G.off_heap) + threadIdx.x;
        for (int i = 0; i < G.HL; ++i) h[i * 128] = kEmpty;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp >= 4 && warp < 8) {
        // ------------------------------------------------------------ producers
        const int pt = threadIdx.x - 128;
        const int nplanes = G.f32 ? 2 : 1;
        const int strip_items = nplanes * G.pw * G.kcols * G.Rb;
        const int norm_items = G.kcols * G.Rb;
        const int* nrm_i = static_cast<const int*>(P.nrm);
        const float* nrm_f = static_cast<const float*>(P.nrm);
        for (int c = 0; c < nchunks; ++c) {
            const int stage = c % kStages, use = c / kStages;
            if (use > 0 && !mbar_wait(bar_empty + 8 * stage, (use - 1) & 1, abort_flag, 1)) break;
            uint8_t* sb = smem + G.off_stage + stage * G.stage_bytes;
            const int jc0 = c * G.kcols;
            const int kc_here = min(G.kcols, NX - jc0);
            for (int t = pt; t < strip_items; t += 128) {
                int r = t;
                const int row = r % G.Rb; r /= G.Rb;
                const int jl = r % G.kcols; r /= G.kcols;
                const int q = r % G.pw;
                const int pl = r / G.pw;
                if (jl >= kc_here) continue;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (row < NR + G.p_eff - 1) {  // rows past that feed no real candidate
                    const uint16_t* plane = pl ? P.plane1 : P.plane0;
                    const uint16_t* prow = plane + (size_t)(Y0 + row) * G.plane_pitch;
                    val = load_shifted16(prow, (X0 + jc0 + jl) * G.Cp + 8 * q);
                }
                *reinterpret_cast<uint4*>(sb + pl * G.plane_stage + q * G.qpitch +
                                          (jl * G.Rb + row) * 16) = val;
            }
            uint8_t* nsb = sb + nplanes * G.plane_stage;
            for (int t = pt; t < norm_items; t += 128) {
                const int row = t % G.Rb, jl = t / G.Rb;
                if (jl >= kc_here) continue;
                uint16_t hi = 0, mid = 0, lo = 0;
                if (row < NR) {
                    const size_t ni = (size_t)(Y0 + row) * G.Wc + (X0 + jc0 + jl);
                    const float w = G.f32 ? nrm_f[ni] : (float)(nrm_i[ni] >> 1);
                    split3(w, hi, mid, lo);
                } else {
                    hi = bf16_bits(1.0e18f);  // no real candidate: never selected
                }
                uint4 val;
                if (G.f32) {
                    val = make_uint4(hi | (uint32_t(mid) << 16), lo | (uint32_t(hi) << 16),
                                     mid | (uint32_t(lo) << 16), 0u);
                } else {
                    val = make_uint4(hi | (uint32_t(mid) << 16), lo, 0u, 0u);
                }
                *reinterpret_cast<uint4*>(nsb + (jl * G.Rb + row) * 16) = val;
            }
            fence_proxy_async();
            mbar_arrive(bar_full + 8 * stage);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t a0 = smem_u32(smem + G.off_a0), a1 = smem_u32(smem + G.off_a1);
            const uint32_t an = smem_u32(smem + G.off_an);
            const uint32_t sbo_a = G.nkc * 128;
            const int nplanes = G.f32 ? 2 : 1;
            const uint32_t lbo_b = G.pw == 1 ? 16u : (uint32_t)G.qpitch;
            int c = 0;
            for (; c < nchunks; ++c) {
                const int stage = c % kStages, use = c / kStages;
                const int buf = c & 1, ub = c >> 1;
                if (ub > 0 && !mbar_wait(bar_tempty + 8 * buf, (ub - 1) & 1, abort_flag, 2)) break;
                if (!mbar_wait(bar_full + 8 * stage, use & 1, abort_flag, 3)) break;
                tc_fence_after();
                const int kc_here = min(G.kcols, NX - c * G.kcols);
                const uint32_t idesc = idesc_bf16(128, kc_here * G.Rb);
                const uint32_t d = tmem_base + buf * kBufCols;
                const uint32_t sb = smem_u32(smem + G.off_stage + stage * G.stage_bytes);
                uint32_t acc = 0;
                for (int t = 0; t < G.nkc / 2; ++t) {
                    const int kc = 2 * t;
                    const int u = kc / G.pw, q = kc % G.pw;
                    const uint32_t boff = q * G.qpitch + u * 16;
                    const uint64_t da0 = sdesc(a0 + kc * 128, 128, sbo_a);
                    const uint64_t db0 = sdesc(sb + boff, lbo_b, 128);
                    mma_bf16(d, da0, db0, idesc, acc);
                    acc = 1;
                    if (nplanes == 2) {
                        const uint64_t db1 = sdesc(sb + G.plane_stage + boff, lbo_b, 128);
                        const uint64_t da1 = sdesc(a1 + kc * 128, 128, sbo_a);
                        mma_bf16(d, da0, db1, idesc, 1);
                        mma_bf16(d, da1, db0, idesc, 1);
                    }
                }
                const uint32_t nsb = sb + nplanes * G.plane_stage;
                mma_bf16(d, sdesc(an, 128, 256), sdesc(nsb, 16, 128), idesc, 1);
                mma_commit(bar_empty + 8 * stage);
                mma_commit(bar_tfull + 8 * buf);
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
        Heap heap{reinterpret_cast<unsigned long long*>(smem + G.off_heap) + threadIdx.x, G.HL};
        const int ry = ry0 + warp, rx = rx0 + lane;
        const bool row_ok = ry < G.n_ry;
        const bool lane_ok = row_ok && rx < G.n_rx;
        const int yr = ry * G.s, xr = rx * G.s;
        const int lo = max(0, yr - G.h - Y0), hi = min(NR - 1, yr + G.h - Y0);
        int nr_i = 0;
        const int* nrm_i = static_cast<const int*>(P.nrm);
        if (lane_ok && !G.f32) nr_i = nrm_i[(size_t)yr * G.Wc + xr];
        float thr = -__int_as_float(0x7f800000);  // -inf while the heap has empty slots
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int c = 0; c < nchunks; ++c) {
            const int buf = c & 1, ub = c >> 1;
            if (!mbar_wait(bar_tfull + 8 * buf, ub & 1, abort_flag, 4)) break;
            tc_fence_after();
            const int jc0 = c * G.kcols;
            const int kc_here = min(G.kcols, NX - jc0);
            if (row_ok) {
                for (int jl = 0; jl < kc_here; ++jl) {
                    const int xc = X0 + jc0 + jl;
                    const bool xok = lane_ok && abs(xc - xr) <= G.h;
                    if (!__any_sync(0xffffffffu, xok)) continue;
                    const uint32_t colbase = tmem_base + lane_base + buf * kBufCols + jl * G.Rb;
                    for (int b = lo >> 4; b <= (hi >> 4); ++b) {
                        float v[16];
                        tmem_ld16(colbase + 16 * b, v);
                        const int i0 = max(lo - 16 * b, 0), i1 = min(hi - 16 * b, 15);
                        float m;
                        if (i0 == 0 && i1 == 15) {
                            float a = max3(v[0], v[1], v[2]), bq = max3(v[3], v[4], v[5]);
                            float cq = max3(v[6], v[7], v[8]), dq = max3(v[9], v[10], v[11]);
                            float e = max3(v[12], v[13], v[14]);
                            m = max3(max3(a, bq, cq), max3(dq, e, v[15]), a);
                        } else {
                            m = -__int_as_float(0x7f800000);
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (i >= i0 && i <= i1) m = fmaxf(m, v[i]);
                        }
                        if (xok && m >= thr) {
                            // slow path: exact keys for every candidate at or above the threshold
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                if (i < i0 || i > i1 || !(v[i] >= thr)) continue;
                                const int yc = Y0 + 16 * b + i;
                                const unsigned off = (unsigned)(yc * G.W + xc);
                                unsigned long long key;
                                if (G.f32) {
                                    key = ((unsigned long long)(~orderable(v[i])) << 32) | off;
                                } else {
                                    const int nc = nrm_i[(size_t)yc * G.Wc + xc];
                                    const int dd = nr_i - 2 * (int)v[i] + (nc & 1);
                                    key = ((unsigned long long)(unsigned)dd << 32) | off;
                                }
                                if (key < heap.top()) {
                                    heap.replace_top(key);
                                    const unsigned long long t = heap.top();
                                    if (t != kEmpty) {
                                        if (G.f32) {
                                            thr = from_orderable(~(unsigned)(t >> 32));
                                        } else {
                                            const int dk = (int)(t >> 32);
                                            thr = (float)((nr_i - dk) >> 1) - 1.0f;
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(bar_tempty + 8 * buf);
        }
        // ---- write results
        if (lane_ok && !*abort_flag) {
            heap.sort();
            const size_t ref = (size_t)ry * G.n_rx + rx;
            if (G.f32) {
                for (int k = 0; k < G.HL; ++k) {
                    const unsigned long long key = heap.h[k * 128];
                    if (key == kEmpty) {
                        P.pool_idx[ref * G.HL + k] = -1;
                        P.pool_score[ref * G.HL + k] = -__int_as_float(0x7f800000);
                    } else {
                        P.pool_idx[ref * G.HL + k] = (int32_t)(unsigned)(key & 0xffffffffu);
                        P.pool_score[ref * G.HL + k] = from_orderable(~(unsigned)(key >> 32));
                    }
                }
            } else {
                for (int k = 0; k < G.K; ++k) {
                    const unsigned long long key = heap.h[k * 128];
                    if (key == kEmpty) {
                        P.out_idx[ref * G.K + k] = -1;
                        P.out_dist[ref * G.K + k] = 0x7fffffff;
                    } else {
                        P.out_idx[ref * G.K + k] = (int32_t)(unsigned)(key & 0xffffffffu);
                        P.out_dist[ref * G.K + k] = (int32_t)(unsigned)(key >> 32);
                    }
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

bool make_tc_geom(const Geom& g, TcGeom& t) {
    t.H = g.H; t.W = g.W; t.Cp = g.Cp; t.p = g.p; t.h = g.h; t.s = g.s; t.K = g.K;
    t.n_ry = g.n_ry; t.n_rx = g.n_rx; t.Hc = g.Hc; t.Wc = g.Wc;
    t.pw = g.pw; t.p_eff = g.p_eff; t.nkc = g.p_eff * g.pw;
    t.f32 = g.dtype == kF32;
    t.HL = t.f32 ? g.L : g.K;
    t.plane_pitch = g.plane_pitch;
    const int nr_max = 3 * g.s + 2 * g.h + 1;
    t.Rb = (nr_max + g.p_eff - 1 + 15) / 16 * 16;
    if (t.Rb > kBufCols) return false;
    t.kcols = kBufCols / t.Rb;
    const int strip_rows = t.kcols * t.Rb + g.p_eff + 16;
    t.qpitch = strip_rows * 16;
    t.plane_stage = t.pw * t.qpitch;
    t.ns_bytes = (t.kcols * t.Rb + 16) * 16;
    const int nplanes = t.f32 ? 2 : 1;
    t.stage_bytes = (nplanes * t.plane_stage + t.ns_bytes + 127) / 128 * 128;
    int off = 0;
    const int a_bytes = 128 * t.nkc * 16;
    t.off_a0 = off; off += a_bytes;
    t.off_a1 = off; off += t.f32 ? a_bytes : 0;
    t.off_an = off; off += 128 * 2 * 16;
    t.off_stage = off; off += kStages * t.stage_bytes;
    t.off_heap = off; off += 128 * t.HL * 8;
    t.off_bar = off; off += (2 * kStages + 5) * 8 + 16;
    t.smem_total = (off + 1023) / 1024 * 1024;
    // the plane padding covers the widest read (see make_geom)
    return t.smem_total <= kSmemLimit;
}

}  // namespace

bool tc_supported(const Geom& g) {
    TcGeom t;
    return make_tc_geom(g, t);
}

cudaError_t launch_tc(const Geom& g, const TcArgs& a, cudaStream_t st) {
    TcParams P{};
    if (!make_tc_geom(g, P.g)) return cudaErrorNotSupported;
    P.plane0 = a.plane0;
    P.plane1 = a.plane1;
    P.nrm = a.nrm;
    P.out_idx = a.out_idx;
    P.out_dist = a.out_dist;
    P.pool_idx = a.pool_idx;
    P.pool_score = a.pool_score;
    P.status = a.status;
    // at least 114 KB of shared memory keeps one CTA per SM (whole-TMEM allocation)
    const int smem = P.g.smem_total < 116 * 1024 ? 116 * 1024 : P.g.smem_total;
    cudaFuncSetAttribute(tc_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 grid((g.n_rx + 31) / 32, (g.n_ry + 3) / 4);
    tc_match_kernel<<<grid, kThreads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace bm
