// ncc.cu -- block matching by normalized cross-correlation (§III-A,
// Eq. equ:cor; Lemma 1 and Theorem 1, case 3: the same ranking is the
// Self-Convolution cross term C_r(j) scaled by g(j) = 1 / (||X_r|| ||X_j||)).
//
// For every reference X_r of the stride grid, the K candidates of its clipped
// search window with the largest
//   ncc(r, j) = <X_r, X_j> / (||X_r||_F ||X_j||_F)
// (the uncentred cosine; a patch of zero norm scores 0), ties broken by the
// smaller row-major offset.  uint8: the cross term a_j and the norm n_j are
// exact integers (float32 sums of integers below 2^24), and a_j / sqrt(n_j)
// is ranked exactly through a_j^2 n_k versus a_k^2 n_j in 128-bit integers,
// so indices are exact.  float32: ranked by the float32 score.
//
// GB300 layout of the work (CUDA cores).  One block per 8 x 8 tile of
// references; the union of the tile's windows is staged in shared memory.
//   Fast path (K <= 32, instantiated patch shapes with p*p*C <= 64): the
//   region is stored as element pairs (pair e of a row holds elements e and
//   e + 1) and read with 64-bit loads.  The norms ||X_j||^2 of all patch
//   positions of the region are formed once per block (they do not depend on
//   the reference) and kept beside it.  One warp per reference, one lane per
//   candidate: the cross term two elements at a time with packed FP32
//   (fma.rn.f32x2), in two chains.  The warp keeps the K best candidates one
//   per lane, in order; a round of 32 new candidates costs one ballot against
//   the K-th, and each candidate that beats it is inserted at its rank
//   (ballot count) with one shuffle of the list.  float32 ranks one 64-bit
//   key per candidate (order-preserving score bits above the offset); uint8
//   keeps (a, n, offset) for its exact comparison.
//   General path: one thread per reference, its K best in a max-heap (worst
//   at the root) in shared memory.
#include "bm.h"
#include "bm_internal.h"

#include <algorithm>
#include <cmath>
#include <string>

namespace bm {
namespace {

constexpr int kNccTile = 8;
constexpr int kNccThreads = kNccTile * kNccTile;
constexpr int kNccMaxK = 64;
constexpr int kNccSmemLimit = 200 * 1024;
constexpr int kNccRows = 4;  // fast path: vertically adjacent candidates per lane

struct NccParams {
    const void* img;
    int32_t* out_idx;  // [n_ry*n_rx][K]
    float* out_score;  // [n_ry*n_rx][K]
    int H, W, C, p, h, s, K, n_ry, n_rx, Hc, Wc, tiles_x;
    int dtype;
};

// Heap entry: cross term and norm (uint8: exact integers; float32: the
// score in `a`, `n` unused) and the candidate offset.
struct Ent {
    float a, n;
    int off;
};

// true if x ranks before y (larger score, then smaller offset)
template <bool kU8>
__device__ __forceinline__ bool better(const Ent& x, const Ent& y) {
    if (x.off < 0 || y.off < 0) return y.off < 0 && x.off >= 0;  // empty slots rank last
    if (kU8) {
        const unsigned long long ax = (unsigned long long)x.a, ay = (unsigned long long)y.a;
        const unsigned long long A = ax * ax, B = ay * ay;
        const unsigned long long nx = (unsigned long long)x.n, ny = (unsigned long long)y.n;
        const unsigned long long h1 = __umul64hi(A, ny), l1 = A * ny;  // a_x^2 n_y
        const unsigned long long h2 = __umul64hi(B, nx), l2 = B * nx;  // a_y^2 n_x
        if (h1 != h2) return h1 > h2;
        if (l1 != l2) return l1 > l2;
    } else {
        if (x.a != y.a) return x.a > y.a;
    }
    return x.off < y.off;
}

// Max-heap of the K best (worst at the root), entry i of thread t at h[i * nthr].
template <bool kU8>
__device__ void heap_push(Ent* h, int nthr, int K, const Ent& e) {
    if (!better<kU8>(e, h[0])) return;
    int i = 0;
    while (true) {
        const int l = 2 * i + 1;
        if (l >= K) break;
        int c = l;
        if (l + 1 < K && better<kU8>(h[l * nthr], h[(l + 1) * nthr])) c = l + 1;  // worse child
        if (!better<kU8>(e, h[c * nthr])) break;  // e is worse than (or as bad as) the worse child: stop
        h[i * nthr] = h[c * nthr];
        i = c;
    }
    h[i * nthr] = e;
}

template <bool kU8>
__global__ void __launch_bounds__(kNccThreads) ncc_kernel(const NccParams Q) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int ty = blockIdx.x / Q.tiles_x, tx = blockIdx.x - ty * Q.tiles_x;
    const int ry0 = ty * kNccTile, rx0 = tx * kNccTile;
    const int ry1 = min(ry0 + kNccTile, Q.n_ry) - 1, rx1 = min(rx0 + kNccTile, Q.n_rx) - 1;
    const int Y0 = max(0, ry0 * Q.s - Q.h), X0 = max(0, rx0 * Q.s - Q.h);
    const int Y1 = min(Q.Hc - 1, ry1 * Q.s + Q.h) + Q.p, X1 = min(Q.Wc - 1, rx1 * Q.s + Q.h) + Q.p;
    const int nrow = Y1 - Y0, pitch = (X1 - X0) * Q.C;
    float* sreg = reinterpret_cast<float*>(smem);
    Ent* heap = reinterpret_cast<Ent*>(smem + (((size_t)nrow * pitch * 4 + 15) & ~size_t(15)));
    for (int i = threadIdx.x; i < nrow * pitch; i += blockDim.x) {
        const int r = i / pitch, e = i - r * pitch;
        const size_t g = ((size_t)(Y0 + r) * Q.W + X0) * Q.C + e;
        sreg[i] = kU8 ? (float)static_cast<const uint8_t*>(Q.img)[g] : static_cast<const float*>(Q.img)[g];
    }
    Ent* h = heap + threadIdx.x;
    for (int i = 0; i < Q.K; ++i) h[i * kNccThreads] = Ent{0.f, 1.f, -1};
    __syncthreads();
    const int ry = ry0 + threadIdx.x / kNccTile, rx = rx0 + threadIdx.x % kNccTile;
    if (ry > ry1 || rx > rx1) return;
    const int yr = ry * Q.s, xr = rx * Q.s, pc = Q.p * Q.C;
    const float* rp = sreg + (yr - Y0) * pitch + (xr - X0) * Q.C;
    float nr = 0.f;
    for (int u = 0; u < Q.p; ++u)
        for (int e = 0; e < pc; ++e) nr = fmaf(rp[u * pitch + e], rp[u * pitch + e], nr);
    const int cy0 = max(0, yr - Q.h), cy1 = min(Q.Hc - 1, yr + Q.h);
    const int cx0 = max(0, xr - Q.h), cx1 = min(Q.Wc - 1, xr + Q.h);
    for (int yc = cy0; yc <= cy1; ++yc) {
        for (int xc = cx0; xc <= cx1; ++xc) {
            const float* cp = sreg + (yc - Y0) * pitch + (xc - X0) * Q.C;
            float a = 0.f, n = 0.f;
            for (int u = 0; u < Q.p; ++u) {
                const float* cr = cp + u * pitch;
                const float* rr = rp + u * pitch;
#pragma unroll 8
                for (int e = 0; e < pc; ++e) {
                    const float c = cr[e];
                    a = fmaf(rr[e], c, a);
                    n = fmaf(c, c, n);
                }
            }
            Ent ent;
            ent.off = yc * Q.W + xc;
            if (kU8) {
                // zero norms score 0
                const bool z = n == 0.f || nr == 0.f;
                ent.a = z ? 0.f : a;
                ent.n = z ? 1.f : n;
            } else {
                ent.a = (n > 0.f && nr > 0.f) ? a * rsqrtf(n) : 0.f;
                ent.n = 1.f;
            }
            heap_push<kU8>(h, kNccThreads, Q.K, ent);
        }
    }
    // heap sort: repeatedly move the root (worst) to the end
    for (int m = Q.K - 1; m > 0; --m) {
        const Ent top = h[0];
        const Ent last = h[m * kNccThreads];
        h[m * kNccThreads] = top;
        // sift `last` down in h[0 .. m)
        int i = 0;
        while (true) {
            const int l = 2 * i + 1;
            if (l >= m) break;
            int c = l;
            if (l + 1 < m && better<kU8>(h[l * kNccThreads], h[(l + 1) * kNccThreads])) c = l + 1;
            if (!better<kU8>(last, h[c * kNccThreads])) break;
            h[i * kNccThreads] = h[c * kNccThreads];
            i = c;
        }
        h[i * kNccThreads] = last;
    }
    // h[0] is now the best, h[K-1] the worst
    const size_t ref = (size_t)ry * Q.n_rx + rx;
    const float inr = nr > 0.f ? rsqrtf(nr) : 0.f;
    for (int k = 0; k < Q.K; ++k) {
        const Ent e = h[k * kNccThreads];
        Q.out_idx[ref * Q.K + k] = e.off;
        float sc = -__int_as_float(0x7f800000);
        if (e.off >= 0) {
            if (kU8) sc = nr > 0.f ? (float)((double)e.a / sqrt((double)nr * (double)e.n)) : 0.f;
            else sc = e.a * inr;
        }
        Q.out_score[ref * Q.K + k] = sc;
    }
}

// ---------------------------------------------------------------- fast path

// An element pair straight from shared memory into a 64-bit register (the
// operand form of the packed FP32 instructions).
__device__ __forceinline__ unsigned long long ld2(const float2* q) {
    return *reinterpret_cast<const unsigned long long*>(q);
}
__device__ __forceinline__ float sum2(unsigned long long v) {
    return __uint_as_float((unsigned)v) + __uint_as_float((unsigned)(v >> 32));
}

template <int P, int C, bool kU8>
__global__ void __launch_bounds__(256) ncc_warp_kernel(const NccParams Q) {
    constexpr int PC = P * C, NPR = PC / 2, TAIL = PC & 1;
    constexpr int R = kNccRows, NW = P + R - 1;
    extern __shared__ __align__(16) float2 sp[];
    const int ty = blockIdx.x / Q.tiles_x, tx = blockIdx.x - ty * Q.tiles_x;
    const int ry0 = ty * kNccTile, rx0 = tx * kNccTile;
    const int ry1 = min(ry0 + kNccTile, Q.n_ry) - 1, rx1 = min(rx0 + kNccTile, Q.n_rx) - 1;
    const int Y0 = max(0, ry0 * Q.s - Q.h), X0 = max(0, rx0 * Q.s - Q.h);
    const int Y1 = min(Q.Hc - 1, ry1 * Q.s + Q.h) + P, X1 = min(Q.Wc - 1, rx1 * Q.s + Q.h) + P;
    // R - 1 zero rows below the region: the last row group of a window reads
    // them for candidates past its end, whose results are dropped
    const int nrow = Y1 - Y0, srow = nrow + R - 1, pitch = (X1 - X0) * C;
    for (int i = threadIdx.x; i < srow * pitch; i += blockDim.x) {
        const int r = i / pitch, e = i - r * pitch;
        float a = 0.f, b = 0.f;
        if (r < nrow) {
            const size_t g = ((size_t)(Y0 + r) * Q.W + X0) * C + e;
            if (kU8) {
                const uint8_t* im = static_cast<const uint8_t*>(Q.img);
                a = im[g];
                b = e + 1 < pitch ? im[g + 1] : 0.f;
            } else {
                const float* im = static_cast<const float*>(Q.img);
                a = im[g];
                b = e + 1 < pitch ? im[g + 1] : 0.f;
            }
        }
        sp[i] = make_float2(a, b);
    }
    __syncthreads();
    // ||X_j||^2 of every patch position of the region, once per block (it
    // does not depend on the reference)
    const int npy = nrow - P + 1, npx = X1 - X0 - P + 1;
    float* snorm = reinterpret_cast<float*>(sp + srow * pitch);
    for (int i = threadIdx.x; i < npy * npx; i += blockDim.x) {
        const int y = i / npx, x = i - y * npx;
        const float2* cb = sp + y * pitch + x * C;
        unsigned long long n2 = 0ull;
        float nt = 0.f;
#pragma unroll
        for (int u = 0; u < P; ++u) {
#pragma unroll
            for (int t = 0; t < NPR; ++t) {
                const unsigned long long c2 = ld2(&cb[u * pitch + 2 * t]);
                asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(n2) : "l"(c2));
            }
            if (TAIL) nt = fmaf(cb[u * pitch + PC - 1].x, cb[u * pitch + PC - 1].x, nt);
        }
        snorm[i] = sum2(n2) + nt;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ntx = rx1 - rx0 + 1, nref = (ry1 - ry0 + 1) * ntx;
    const int K = Q.K;
    for (int rl = warp; rl < nref; rl += nwarps) {
        const int ry = ry0 + rl / ntx, rx = rx0 + rl % ntx;
        const int yr = ry * Q.s, xr = rx * Q.s;
        const float2* rb = sp + (yr - Y0) * pitch + (xr - X0) * C;
        const float nr = snorm[(yr - Y0) * npx + (xr - X0)];
        const int cy0 = max(0, yr - Q.h), cy1 = min(Q.Hc - 1, yr + Q.h);
        const int cx0 = max(0, xr - Q.h), cx1 = min(Q.Wc - 1, xr + Q.h);
        const int wx = cx1 - cx0 + 1;
        const int nitem = ((cy1 - cy0 + R) / R) * wx;  // (row group, column)
        // cross terms <X_r, X_j> of the R candidates (yc + i, xc), i < R: each
        // window row loaded serves up to R of them, the reference by broadcast
        auto cross = [&](int yc, int xc, float (&a)[R]) {
            const float2* cb = sp + (yc - Y0) * pitch + (xc - X0) * C;
            unsigned long long a2[R];
            float at[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                a2[i] = 0ull;
                at[i] = 0.f;
            }
#pragma unroll
            for (int t = 0; t < NPR; ++t) {
                unsigned long long w[NW];
#pragma unroll
                for (int u = 0; u < NW; ++u) w[u] = ld2(&cb[u * pitch + 2 * t]);
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    const unsigned long long r2 = ld2(&rb[u * pitch + 2 * t]);
#pragma unroll
                    for (int i = 0; i < R; ++i)
                        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a2[i]) : "l"(r2), "l"(w[u + i]));
                }
            }
            if (TAIL) {
                float w[NW];
#pragma unroll
                for (int u = 0; u < NW; ++u) w[u] = cb[u * pitch + PC - 1].x;
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    const float rv = rb[u * pitch + PC - 1].x;
#pragma unroll
                    for (int i = 0; i < R; ++i) at[i] = fmaf(rv, w[u + i], at[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = sum2(a2[i]) + at[i];
        };
        const size_t ref = (size_t)ry * Q.n_rx + rx;
        if constexpr (!kU8) {
            // float32: the rank is (score, offset), one 64-bit key per candidate,
            // smaller is better: the score's order-preserving bits, complemented,
            // above the offset
            unsigned long long mine = ~0ull, kth = ~0ull;
            for (int j0 = 0; j0 < nitem; j0 += 32) {
                const int j = j0 + lane;
                const bool live = j < nitem;
                float a[R];
                int yc = cy0, xc = cx0;
                if (live) {
                    const int jb = j / wx;
                    yc = cy0 + jb * R;
                    xc = cx0 + j - jb * wx;
                    cross(yc, xc, a);
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    unsigned long long key = ~0ull;
                    if (live && yc + i <= cy1) {
                        const float n = snorm[(yc + i - Y0) * npx + (xc - X0)];
                        // + 0.f makes a zero score +0 (-0 would order below it)
                        const float sc = ((n > 0.f && nr > 0.f) ? a[i] * rsqrtf(n) : 0.f) + 0.f;
                        const unsigned b = __float_as_uint(sc);
                        const unsigned ord = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
                        key = ((unsigned long long)~ord << 32) | (unsigned)((yc + i) * Q.W + xc);
                    }
                    warp_list_offer(key, mine, kth, lane, K);
                }
            }
            if (lane < K) {
                float sc = -__int_as_float(0x7f800000);
                int off = -1;
                if (mine != ~0ull) {
                    const unsigned ord = ~(unsigned)(mine >> 32);
                    const float s = __uint_as_float((ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord);
                    sc = nr > 0.f ? s * rsqrtf(nr) : 0.f;
                    off = (int)(unsigned)mine;
                }
                Q.out_idx[ref * K + lane] = off;
                Q.out_score[ref * K + lane] = sc;
            }
        } else {
            // uint8: exact ranking through a^2 n products, (a, n, offset) per entry
            Ent mine{0.f, 1.f, -1};  // entry `lane` in rank order (lanes >= K: nothing of use)
            Ent kth{0.f, 1.f, -1};
            for (int j0 = 0; j0 < nitem; j0 += 32) {
                const int j = j0 + lane;
                const bool live = j < nitem;
                float a[R];
                int yc = cy0, xc = cx0;
                if (live) {
                    const int jb = j / wx;
                    yc = cy0 + jb * R;
                    xc = cx0 + j - jb * wx;
                    cross(yc, xc, a);
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    Ent c{0.f, 1.f, -1};
                    if (live && yc + i <= cy1) {
                        const float n = snorm[(yc + i - Y0) * npx + (xc - X0)];
                        c.off = (yc + i) * Q.W + xc;
                        const bool z = n == 0.f || nr == 0.f;
                        c.a = z ? 0.f : a[i];
                        c.n = z ? 1.f : n;
                    }
                    unsigned mask = __ballot_sync(0xffffffffu, c.off >= 0 && better<true>(c, kth));
                    while (mask) {
                        const int src = __ffs(mask) - 1;
                        mask &= mask - 1;
                        Ent b;
                        b.a = __shfl_sync(0xffffffffu, c.a, src);
                        b.n = __shfl_sync(0xffffffffu, c.n, src);
                        b.off = __shfl_sync(0xffffffffu, c.off, src);
                        if (!better<true>(b, kth)) continue;  // the K-th moved past it
                        const int pos = __popc(__ballot_sync(0xffffffffu, lane < K && better<true>(mine, b)));
                        Ent up;
                        up.a = __shfl_up_sync(0xffffffffu, mine.a, 1);
                        up.n = __shfl_up_sync(0xffffffffu, mine.n, 1);
                        up.off = __shfl_up_sync(0xffffffffu, mine.off, 1);
                        if (lane == pos) mine = b;
                        else if (lane > pos) mine = up;
                        kth.a = __shfl_sync(0xffffffffu, mine.a, K - 1);
                        kth.n = __shfl_sync(0xffffffffu, mine.n, K - 1);
                        kth.off = __shfl_sync(0xffffffffu, mine.off, K - 1);
                    }
                }
            }
            if (lane < K) {
                float sc = -__int_as_float(0x7f800000);
                if (mine.off >= 0)
                    sc = nr > 0.f ? (float)((double)mine.a / sqrt((double)nr * (double)mine.n)) : 0.f;
                Q.out_idx[ref * K + lane] = mine.off;
                Q.out_score[ref * K + lane] = sc;
            }
        }
    }
}


// ---------------------------------------------------------------- tensor-core form

// The tensor-core kernel in its NCC mode (uncentred operands, no norm K-step,
// each value scaled by 1 / ||X_j|| in the epilogue) leaves per reference a
// pool of the L best approximate scores s~_j = a~_j / ||X_j|| (a~_j the
// tensor-core cross term: exact for uint8, the bf16 hi/lo split for float32,
// |a~_j - a_j| <= eps ||X_r|| ||X_j||; 32-bit pool keys round s~ up by less
// than round_rel relative).  This kernel ranks the pool exactly -- uint8
// through (a, n) integer products as the CUDA-core kernels do, float32 by the
// float32 score of a direct cross term -- and keeps the pool's top K when no
// candidate outside it can reach them: the K-th exact pool score must exceed
// the pool's last approximate score plus the estimate's error bound.  Else
// (or when the pool is full of ties) the reference's whole window is ranked
// directly.  One warp per reference.

struct NccPoolParams {
    const void* img;
    const void* nrm;          // uncentred norms [Hc][Wc] (uint8: int32, float32: float)
    const int32_t* pool_idx;  // [nR][L], best first
    const float* pool_score;
    int32_t* out_idx;
    float* out_score;
    unsigned long long* counters;  // [0] overflow
    int H, W, C, p, h, s, K, L, n_ry, n_rx, Hc, Wc, u8;
    float eps;                // float32 cross-term bound (relative to ||X_r|| ||X_j||)
    float round_rel;          // pool-score rounding (relative)
};

// Exact (uint8) or float32 cross term <X_r, X_j> and ||X_j||^2 from global memory.
template <bool kU8>
__device__ __forceinline__ float cross_term(const NccPoolParams& Q, int yr, int xr, int yc, int xc) {
    const int pc = Q.p * Q.C;
    float a = 0.f;
    for (int u = 0; u < Q.p; ++u) {
        const size_t r0 = ((size_t)(yr + u) * Q.W + xr) * Q.C, c0 = ((size_t)(yc + u) * Q.W + xc) * Q.C;
        for (int e = 0; e < pc; ++e) {
            float x, y;
            if (kU8) {
                x = __ldg(static_cast<const uint8_t*>(Q.img) + r0 + e);
                y = __ldg(static_cast<const uint8_t*>(Q.img) + c0 + e);
            } else {
                x = __ldg(static_cast<const float*>(Q.img) + r0 + e);
                y = __ldg(static_cast<const float*>(Q.img) + c0 + e);
            }
            a = fmaf(x, y, a);
        }
    }
    return a;
}

__device__ __forceinline__ float norm_at(const NccPoolParams& Q, bool u8, int y, int x) {
    const size_t o = (size_t)y * Q.Wc + x;
    return u8 ? (float)__ldg(static_cast<const int*>(Q.nrm) + o) : __ldg(static_cast<const float*>(Q.nrm) + o);
}

// float32 key: smaller is better (complemented order-preserving score bits above the offset)
__device__ __forceinline__ unsigned long long score_key(float sc, int off) {
    sc += 0.f;  // -0 -> +0
    const unsigned b = __float_as_uint(sc);
    const unsigned ord = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)~ord << 32) | (unsigned)off;
}
__device__ __forceinline__ float key_score(unsigned long long k) {
    const unsigned ord = ~(unsigned)(k >> 32);
    return __uint_as_float((ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord);
}

// uint8: entry c offered to the warp's exact list (lane i = rank i < K).
__device__ __forceinline__ void ent_list_offer(const Ent& c, Ent& mine, Ent& kth, int lane, int K) {
    unsigned mask = __ballot_sync(0xffffffffu, c.off >= 0 && better<true>(c, kth));
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        Ent b;
        b.a = __shfl_sync(0xffffffffu, c.a, src);
        b.n = __shfl_sync(0xffffffffu, c.n, src);
        b.off = __shfl_sync(0xffffffffu, c.off, src);
        if (!better<true>(b, kth)) continue;  // the K-th moved past it
        const int pos = __popc(__ballot_sync(0xffffffffu, lane < K && better<true>(mine, b)));
        Ent up;
        up.a = __shfl_up_sync(0xffffffffu, mine.a, 1);
        up.n = __shfl_up_sync(0xffffffffu, mine.n, 1);
        up.off = __shfl_up_sync(0xffffffffu, mine.off, 1);
        if (lane == pos) mine = b;
        else if (lane > pos) mine = up;
        kth.a = __shfl_sync(0xffffffffu, mine.a, K - 1);
        kth.n = __shfl_sync(0xffffffffu, mine.n, K - 1);
        kth.off = __shfl_sync(0xffffffffu, mine.off, K - 1);
    }
}

template <bool kU8>
__global__ void __launch_bounds__(128) ncc_pool_kernel(const __grid_constant__ NccPoolParams Q) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t r = (size_t)blockIdx.x * 4 + warp;
    if (r >= (size_t)Q.n_ry * Q.n_rx) return;  // whole warp
    const int ry = (int)(r / Q.n_rx), rx = (int)(r % Q.n_rx);
    const int yr = ry * Q.s, xr = rx * Q.s;
    const float nr = norm_at(Q, kU8, yr, xr);
    const int K = Q.K;
    // the pool, in order; entry L - 1 present means the pool is full
    Ent mine{0.f, 1.f, -1}, kth{0.f, 1.f, -1};
    unsigned long long mk = ~0ull, kk = ~0ull;
    bool full = false;
    float last = 0.f;  // the pool's last (worst) approximate score, rounded up
    for (int i0 = 0; i0 < Q.L; i0 += 32) {
        const int i = i0 + lane;
        const int off = i < Q.L ? __ldg(Q.pool_idx + r * Q.L + i) : -1;
        if (i == Q.L - 1 && off >= 0) {
            full = true;
            last = __ldg(Q.pool_score + r * Q.L + i);
        }
        int yc = 0, xc = 0;
        float a = 0.f, n = 1.f;
        if (off >= 0) {
            yc = off / Q.W;
            xc = off - yc * Q.W;
            a = cross_term<kU8>(Q, yr, xr, yc, xc);
            n = norm_at(Q, kU8, yc, xc);
        }
        if (kU8) {
            Ent c{0.f, 1.f, off};
            if (off >= 0 && n != 0.f && nr != 0.f) {
                c.a = a;
                c.n = n;
            }
            ent_list_offer(c, mine, kth, lane, K);
        } else {
            const unsigned long long key =
                off >= 0 ? score_key((n > 0.f && nr > 0.f) ? a * rsqrtf(n) : 0.f, off) : ~0ull;
            warp_list_offer(key, mk, kk, lane, K);
        }
    }
    full = __any_sync(0xffffffffu, full);
    last = __shfl_sync(0xffffffffu, last, (Q.L - 1) & 31);
    // can a candidate outside the pool reach the exact top K?
    bool overflow = false;
    if (full) {
        // outside candidates: approximate score <= last, exact score <= last + bound
        if (kU8) {
            const double sK = kth.off < 0 ? -1.0 : (kth.n > 0.f ? (double)kth.a / sqrt((double)kth.n) : 0.0);
            const double lim = (double)last * (1.0 + 2.0 * Q.round_rel) + fabs((double)last) * 1e-6 + 1e-30;
            overflow = !(sK > lim);
        } else {
            const float sK = kk == ~0ull ? -__int_as_float(0x7f800000) : key_score(kk);
            const float bound = Q.eps * sqrtf(fmaxf(nr, 0.f)) + fabsf(last) * 1e-5f + 1e-30f;
            overflow = !(sK > last + bound);
        }
    }
    if (overflow) {
        if (lane == 0) atomicAdd(Q.counters, 1ull);
        // the whole window, directly
        mine = Ent{0.f, 1.f, -1};
        kth = Ent{0.f, 1.f, -1};
        mk = kk = ~0ull;
        const int cy0 = max(0, yr - Q.h), cy1 = min(Q.Hc - 1, yr + Q.h);
        const int cx0 = max(0, xr - Q.h), cx1 = min(Q.Wc - 1, xr + Q.h);
        const int wx = cx1 - cx0 + 1, total = (cy1 - cy0 + 1) * wx;
        for (int j0 = 0; j0 < total; j0 += 32) {
            const int j = j0 + lane;
            int off = -1;
            float a = 0.f, n = 1.f;
            if (j < total) {
                const int yc = cy0 + j / wx, xc = cx0 + j % wx;
                off = yc * Q.W + xc;
                a = cross_term<kU8>(Q, yr, xr, yc, xc);
                n = norm_at(Q, kU8, yc, xc);
            }
            if (kU8) {
                Ent c{0.f, 1.f, off};
                if (off >= 0 && n != 0.f && nr != 0.f) {
                    c.a = a;
                    c.n = n;
                }
                ent_list_offer(c, mine, kth, lane, K);
            } else {
                const unsigned long long key =
                    off >= 0 ? score_key((n > 0.f && nr > 0.f) ? a * rsqrtf(n) : 0.f, off) : ~0ull;
                warp_list_offer(key, mk, kk, lane, K);
            }
        }
    }
    if (lane < K) {
        float sc = -__int_as_float(0x7f800000);
        int off = -1;
        if (kU8) {
            off = mine.off;
            if (off >= 0) sc = nr > 0.f ? (float)((double)mine.a / sqrt((double)nr * (double)mine.n)) : 0.f;
        } else if (mk != ~0ull) {
            off = (int)(unsigned)mk;
            sc = nr > 0.f ? key_score(mk) * rsqrtf(nr) : 0.f;
        }
        Q.out_idx[r * K + lane] = off;
        Q.out_score[r * K + lane] = sc;
    }
}

using NccKernel = void (*)(NccParams);

NccKernel pick_fast(int p, int C, bool u8) {
#define BM_NCC_CASE(PP, CC) \
    if (p == PP && C == CC) return u8 ? ncc_warp_kernel<PP, CC, true> : ncc_warp_kernel<PP, CC, false>;
    BM_NCC_CASE(1, 1) BM_NCC_CASE(2, 1) BM_NCC_CASE(3, 1) BM_NCC_CASE(4, 1) BM_NCC_CASE(5, 1)
    BM_NCC_CASE(6, 1) BM_NCC_CASE(7, 1) BM_NCC_CASE(8, 1)
    BM_NCC_CASE(2, 2) BM_NCC_CASE(3, 2) BM_NCC_CASE(4, 2)
    BM_NCC_CASE(2, 3) BM_NCC_CASE(3, 3) BM_NCC_CASE(4, 3)
    BM_NCC_CASE(2, 4) BM_NCC_CASE(3, 4) BM_NCC_CASE(4, 4)
#undef BM_NCC_CASE
    return nullptr;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};


// The tensor-core form: uncentred planes and norms (1 / ||X_j|| in the
// split-norm slots), the tensor-core kernel in its NCC mode writing a pool of
// L per reference, then ncc_pool_kernel.  Workspace from the context.
int ncc_tensor_core(bm_ctx* ctx, const Geom& g, const void* img, int32_t* out_idx, float* out_score,
                    cudaStream_t st) {
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t b_plane = al(plane_bytes(g)), b_nrm = al(nrm_bytes(g)), b_nsp = al(nsp_bytes(g));
    const size_t b_pool = al((size_t)g.nR * g.L * 4);
    const size_t total = 2 * b_plane + b_nrm + b_nsp + 2 * b_pool + 256;
    void* ws = nullptr;
    int rc = ctx_workspace(ctx, st, total, &ws);
    if (rc != BM_OK) return rc;
    char* b = static_cast<char*>(ws);
    uint16_t* p0 = reinterpret_cast<uint16_t*>(b);
    uint16_t* p1 = reinterpret_cast<uint16_t*>(b + b_plane);
    void* nrm = b + 2 * b_plane;
    uint16_t* nsp = reinterpret_cast<uint16_t*>(b + 2 * b_plane + b_nrm);
    int32_t* pidx = reinterpret_cast<int32_t*>(b + 2 * b_plane + b_nrm + b_nsp);
    float* pscore = reinterpret_cast<float*>(b + 2 * b_plane + b_nrm + b_nsp + b_pool);
    char* hdr = b + 2 * b_plane + b_nrm + b_nsp + 2 * b_pool;
    int* status = reinterpret_cast<int*>(hdr);
    float* center = reinterpret_cast<float*>(hdr + 16);
    PrepJob pj = make_prep_job(g, img, center, p0, p1, nrm, nsp);
    pj.status = status;
    cudaError_t e;
    if ((e = launch_center_batch(&pj, 1, st)) != cudaSuccess || (e = launch_planes_batch(&pj, 1, st)) != cudaSuccess ||
        (e = launch_box_batch(&pj, 1, st)) != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("ncc preparation: ") + cudaGetErrorString(e)).c_str());
    TcArgs a{};
    a.plane0 = p0;
    a.plane1 = p1;
    a.nrm = nrm;
    a.nsp = nsp;
    a.pool_idx = pidx;
    a.pool_score = pscore;
    a.status = status;
    a.fault = ctx_fault_word(ctx);
    if ((e = launch_tc_batch(&g, &a, 1, st)) != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("ncc tensor-core launch: ") + cudaGetErrorString(e)).c_str());
    NccPoolParams Q{};
    Q.img = img; Q.nrm = nrm; Q.pool_idx = pidx; Q.pool_score = pscore;
    Q.out_idx = out_idx; Q.out_score = out_score; Q.counters = ctx_counters(ctx);
    Q.H = g.H; Q.W = g.W; Q.C = g.C; Q.p = g.p; Q.h = g.h; Q.s = g.s; Q.K = g.K; Q.L = g.L;
    Q.n_ry = g.n_ry; Q.n_rx = g.n_rx; Q.Hc = g.Hc; Q.Wc = g.Wc; Q.u8 = g.dtype == kU8;
    Q.eps = 6.103515625e-05f;  // 2^-14: the split cross term's bound, as in block matching
    const int tb = tc_score_bits(g);
    Q.round_rel = tb ? ldexpf(1.0f, tb - 23) : 0.0f;
    const unsigned blocks = (unsigned)((g.nR + 3) / 4);
    if (Q.u8) ncc_pool_kernel<true><<<blocks, 128, 0, st>>>(Q);
    else ncc_pool_kernel<false><<<blocks, 128, 0, st>>>(Q);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("ncc pool launch: ") + cudaGetErrorString(e)).c_str());
    ctx_count_tc_job(ctx);
    return BM_OK;
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

int bm_match_ncc(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                 int window, int stride, int K, int32_t* out_idx, float* out_score,
                 bm_stream stream) {
    if (!ctx) return set_error(BM_ERR_INVALID, "null context");
    if (dtype != BM_U8 && dtype != BM_F32) return set_error(BM_ERR_INVALID, "unknown dtype");
    if (H < 1 || W < 1 || C < 1 || C > kMaxC || patch < 1 || patch > H || patch > W ||
        window < 1 || window % 2 == 0 || window > kMaxWindow || stride < 1 || K < 1 || K > kMaxK)
        return set_error(BM_ERR_INVALID, "invalid geometry or K");
    if (!img || !out_idx || !out_score) return set_error(BM_ERR_INVALID, "null pointer");
    if ((long long)H * W >= (1LL << 31)) return set_error(BM_ERR_UNSUPPORTED, "H*W must be below 2^31");
    if (patch * patch * C > kMaxPatchElems)
        return set_error(BM_ERR_UNSUPPORTED, "patch*patch*C must be at most 256");
    if (K > kNccMaxK) return set_error(BM_ERR_UNSUPPORTED, "K must be at most 64 for NCC");
    DevGuard dg0(ctx_device(ctx));
    if (dtype == BM_U8) {
        // the tensor-core form (uint8, K <= 32, the class fits the kernel).
        // float32 stays on the CUDA-core kernels: its tensor-core form needs
        // the three-product split and a direct re-rank of the pool, and
        // measured slower (687 against 378 us per 512 x 512 image)
        Geom g;
        if (make_geom(g, H, W, C, (int)dtype, patch, window, stride, K) == BM_OK) {
            g.ncc = 1;
            // a pool of 32 (one entry per lane) or K + 8: NCC scores cluster near the top
            g.L = std::min(160, std::max(32, (K + 8 + 7) / 8 * 8));
            if (K <= 32 && ctx_uses_tc(ctx) && tc_supported(g))
                return ncc_tensor_core(ctx, g, img, out_idx, out_score, reinterpret_cast<cudaStream_t>(stream));
        }
    }
    NccParams Q{};
    Q.img = img; Q.out_idx = out_idx; Q.out_score = out_score;
    Q.H = H; Q.W = W; Q.C = C; Q.p = patch; Q.h = (window - 1) / 2; Q.s = stride; Q.K = K;
    Q.n_ry = (H - patch) / stride + 1; Q.n_rx = (W - patch) / stride + 1;
    Q.Hc = H - patch + 1; Q.Wc = W - patch + 1;
    Q.dtype = dtype == BM_U8 ? kU8 : kF32;
    Q.tiles_x = (Q.n_rx + kNccTile - 1) / kNccTile;
    const int tiles = ((Q.n_ry + kNccTile - 1) / kNccTile) * Q.tiles_x;
    const int rows = std::min(H, (kNccTile - 1) * stride + 2 * Q.h + patch);
    const int cols = std::min(W, (kNccTile - 1) * stride + 2 * Q.h + patch);
    const size_t region = (size_t)rows * cols * C;
    // fast path: the region as element pairs, then the norms of its patch positions
    const size_t fast_bytes = (size_t)(rows + kNccRows - 1) * cols * C * sizeof(float2) +
                              (size_t)(rows - patch + 1) * (cols - patch + 1) * sizeof(float);
    NccKernel fast = K <= 32 ? pick_fast(patch, C, Q.dtype == kU8) : nullptr;
    if (fast && fast_bytes > (size_t)kNccSmemLimit) fast = nullptr;
    const size_t smem = fast ? fast_bytes
                             : ((region * 4 + 15) & ~size_t(15)) + (size_t)K * kNccThreads * sizeof(Ent);
    if (smem > (size_t)kNccSmemLimit)
        return set_error(BM_ERR_UNSUPPORTED, "search region does not fit in shared memory");
    DevGuard dg(ctx_device(ctx));
    NccKernel kern = fast ? fast : (Q.dtype == kU8 ? ncc_kernel<true> : ncc_kernel<false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        kern<<<tiles, fast ? 256 : kNccThreads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(Q);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("ncc launch: ") + cudaGetErrorString(e)).c_str());
    return BM_OK;
}

}  // extern "C"
