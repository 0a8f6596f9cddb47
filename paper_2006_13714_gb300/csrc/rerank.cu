// rerank.cu -- (a6) float32 boundary re-rank.
//
// The tensor-core pass leaves, per reference r, a pool of the L largest
// v_j = b~_j + eps n_j (b~ the split-bf16 estimate of Theorem 1's score
// b_j = C_r(j) - 0.5 n_j of the centred patches, n_j = ||X_j - c||^2,
// eps = 2^-14), best first.  The identity d = ||X_r||^2 - 2 b (Lemma 2)
// loses precision to cancellation in proportion to n_r + n_j, not to d, so
// the final distances are recomputed here directly:
//
//   1. Error bound: |b~_j - b_j| <= eps (n_r + n_j).  At least K pool
//      entries have b >= T' = v_K - eps n_r - 2 eps max_{rank<K} n_k, so only
//      entries with u_j = v_j + eps n_r >= T' can be among the K nearest (the
//      band).  If the pool is full and every entry is in the band,
//      candidates outside the pool might qualify too ("overflow"): that
//      reference is recomputed over its whole window.  When the pool scores
//      arrive rounded up (v'_j >= v_j, by less than 2^tbits ulp: the 32-bit
//      keys of the tensor-core pass), T' also subtracts that rounding of the
//      top-K entries.
//   2. Band members get the explicit FP32 distance sum (X_r - X_j)^2
//      (Eq. equ:bmMetric_app), relative error <= gamma = (n + 3) 2^-24 with
//      n = p*p*C terms, and are ranked by (distance, row-major offset).
//   3. If the K-th and (K+1)-th FP32 distances are within that error of each
//      other, the members near the boundary are recomputed in FP64 and their
//      order there follows the FP64 values.
//   4. Counter: band members whose identity estimate misses the direct
//      distance by more than the bound (expected 0).
//
// Layout of the work: one block per tile of TRY x TRX references of one
// image (a table of images per launch).  The block first stages the image
// region its references' windows cover, and the norms there, in shared
// memory, so every distance reads shared memory.  The region is stored as
// element pairs (pair e of a row holds elements e and e + 1), so a patch row
// that starts anywhere is read with 64-bit loads and its squared differences
// are summed two at a time with packed FP32 arithmetic.  One warp per
// reference; every ranking uses 64-bit integer keys (FP64 is slow on this
// part and is kept to the rare boundary ties).  The block's overflow
// references are done last by all its warps together: the (K+1)-th smallest
// key U among the pool's direct distances bounds the keys of the window's
// K+1 nearest, so the warps scan interleaved shares of the window and keep
// only keys <= U (typically little more than K+1 of them), which are then
// ranked like a band.  Should ties leave more than a buffer's worth, one
// warp takes the window's exact top-(K+1) by insertion.  Shapes whose region
// does not fit run the same steps on global memory, one image per launch.
#include "bm_internal.h"

#include <climits>
#include <type_traits>

namespace bm {
namespace {

constexpr float kEps = 6.103515625e-05f;  // 2^-14, same constant as the tensor-core pass
constexpr int kFbSlots = (kMaxK + 1 + 31) / 32;
constexpr unsigned long long kNone = ~0ull;
constexpr int kTileWarps = 8;
constexpr int kMaxTileRefs = 64;
constexpr int kCandCap = kFbSlots * 32;  // window keys kept per overflow reference
constexpr int kMaxRerankJobs = 64;
constexpr int kTileSmemLimit = 220 * 1024;  // within the 227 KB a block may use

struct RerankJob {
    const float* img;
    const float* nrm;
    const int32_t* pool_idx;
    const float* pool_score;
    int32_t* out_idx;
    float* out_dist;
    int H, W, n_ry, n_rx, Hc, Wc;
    FastDiv wdiv;  // offset -> row
    int tiles_x, tile_begin;
};

struct RerankParams {
    int C, p, h, s, K, L;
    float round_rel;  // pool-score rounding, relative: 2^(tbits - 23) (0: exact scores)
    float gamma;      // FP32 relative error bound of a direct distance
    int TRY, TRX;     // references per tile (rows, columns)
    int img_cap;      // shared-memory image region capacity (element pairs); norms follow
    unsigned long long* counters;  // [0] overflow, [1] fp64 rechecks, [2] bound violations
    int njobs, total_tiles;
    RerankJob jobs[kMaxRerankJobs];
};

// Pixel sources; element (y, x, c) of the image at elem(at(y, x), c).
// PairSrc: a region in shared memory as element pairs {X[e], X[e + 1]}.
struct PairSrc {
    const float2* base;
    int y0, x0, pitch, C;
    __device__ __forceinline__ const float2* at(int y, int x) const {
        return base + (y - y0) * pitch + (x - x0) * C;
    }
    __device__ __forceinline__ static float elem(const float2* row, int e) { return row[e].x; }
};
// QuadSrc: a region in shared memory stored plainly, for C a multiple of 4:
// every patch row starts on a 16-byte boundary and is read as float4.
struct QuadSrc {
    const float* base;
    int y0, x0, pitch, C;
    __device__ __forceinline__ const float* at(int y, int x) const {
        return base + (y - y0) * pitch + (x - x0) * C;
    }
    __device__ __forceinline__ static float elem(const float* row, int e) { return row[e]; }
};
// PlainSrc: the image in global memory, or the norms region.
struct PlainSrc {
    const float* base;
    int y0, x0, pitch, C;
    __device__ __forceinline__ const float* at(int y, int x) const {
        return base + (size_t)(y - y0) * pitch + (size_t)(x - x0) * C;
    }
    __device__ __forceinline__ static float elem(const float* row, int e) { return row[e]; }
};

__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}

// (X_r - X_j)^2 summed over the patch (the reference's rows at
// ref + u * pitch): elements two at a time with packed FP32 subtract and
// fused multiply-add, even and odd elements in two running sums.  FP, FC:
// the patch side and channels when fixed at compile time (0: runtime p, C),
// which unrolls the sum completely.
template <int FP = 0, int FC = 0>
__device__ __forceinline__ float direct_f32(const PairSrc& X, int p_rt, int C_rt, const float2* ref,
                                            int yc, int xc) {
    const int p = FP ? FP : p_rt, C = FC ? FC : C_rt;
    const int pc = p * C, np = pc >> 1;
    // two packed running sums (even and odd patch rows) halve the dependent chain
    unsigned long long acc[2] = {0ull, 0ull};
    float tail = 0.f;
    const float2* cbase = X.at(yc, xc);
#pragma unroll
    for (int u = 0; u < p; ++u) {
        const float2* crow = cbase + u * X.pitch;
        const float2* rrow = ref + u * X.pitch;
#pragma unroll 4
        for (int t = 0; t < np; ++t) {
            unsigned long long d;
            asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(rrow[2 * t])), "l"(f2_bits(crow[2 * t])));
            asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc[u & 1]) : "l"(d));
        }
        if (pc & 1) {
            const float d = rrow[pc - 1].x - crow[pc - 1].x;
            tail = fmaf(d, d, tail);
        }
    }
    return ((__uint_as_float((unsigned)acc[0]) + __uint_as_float((unsigned)(acc[0] >> 32))) +
            (__uint_as_float((unsigned)acc[1]) + __uint_as_float((unsigned)(acc[1] >> 32)))) + tail;
}

// The same sum from a QuadSrc region: four elements per 16-byte load, two
// packed subtract / fused multiply-add pairs, four running sums.
template <int FP = 0, int FC = 0>
__device__ __forceinline__ float direct_f32(const QuadSrc& X, int p_rt, int C_rt, const float* ref,
                                            int yc, int xc) {
    const int p = FP ? FP : p_rt, C = FC ? FC : C_rt;
    const int nq = (p * C) >> 2;  // float4 per patch row
    unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
    const float* cbase = X.at(yc, xc);
#pragma unroll
    for (int u = 0; u < p; ++u) {
        const float4* crow = reinterpret_cast<const float4*>(cbase + u * X.pitch);
        const float4* rrow = reinterpret_cast<const float4*>(ref + u * X.pitch);
#pragma unroll 4
        for (int t = 0; t < nq; ++t) {
            const float4 a = rrow[t], b = crow[t];
            unsigned long long d0, d1;
            asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(f2_bits(make_float2(a.x, a.y))), "l"(f2_bits(make_float2(b.x, b.y))));
            asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(f2_bits(make_float2(a.z, a.w))), "l"(f2_bits(make_float2(b.z, b.w))));
            asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc[2 * (u & 1)]) : "l"(d0));
            asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc[2 * (u & 1) + 1]) : "l"(d1));
        }
    }
    auto lo = [](unsigned long long v) { return __uint_as_float((unsigned)v); };
    auto hi = [](unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); };
    return ((lo(acc[0]) + hi(acc[0])) + (lo(acc[1]) + hi(acc[1]))) +
           ((lo(acc[2]) + hi(acc[2])) + (lo(acc[3]) + hi(acc[3])));
}

// The same sum elementwise in order (global-memory source).
__device__ __forceinline__ float direct_f32(const PlainSrc& X, int p, int C, const float* ref,
                                            int yc, int xc) {
    const int pc = p * C;
    float acc = 0.f;
    for (int u = 0; u < p; ++u) {
        const float* crow = X.at(yc + u, xc);
        const float* rrow = ref + (size_t)u * X.pitch;
#pragma unroll 8
        for (int e = 0; e < pc; ++e) {
            const float d = rrow[e] - crow[e];
            acc = fmaf(d, d, acc);
        }
    }
    return acc;
}

template <class Src, class T>
__device__ __forceinline__ double direct_f64(const Src& X, int p, int C, const T* ref, int yc, int xc) {
    const int pc = p * C;
    double acc = 0.0;
    for (int u = 0; u < p; ++u) {
        const T* crow = X.at(yc + u, xc);
        const T* rrow = ref + (size_t)u * X.pitch;
        for (int e = 0; e < pc; ++e) {
            const double d = (double)Src::elem(rrow, e) - (double)Src::elem(crow, e);
            acc = fma(d, d, acc);
        }
    }
    return acc;
}

// rank[i] = number of keys (over all 32*S lane-strided slots) smaller than key[i].
// Empty slots (kNone) are never smaller than a key, so each slot's scan stops
// at its last lane that holds one.
template <int S>
__device__ __forceinline__ void warp_rank(const unsigned long long (&key)[S], int (&rank)[S]) {
#pragma unroll
    for (int i = 0; i < S; ++i) rank[i] = 0;
#pragma unroll
    for (int slot = 0; slot < S; ++slot) {
        const int nsrc = 32 - __clz((int)__ballot_sync(0xffffffffu, key[slot] != kNone));
        for (int src = 0; src < nsrc; ++src) {
            const unsigned long long km = __shfl_sync(0xffffffffu, key[slot], src);
#pragma unroll
            for (int i = 0; i < S; ++i) rank[i] += km < key[i] ? 1 : 0;
        }
    }
}

// One key per lane: odd-even transposition steps (lane pairs exchange
// out-of-order keys) until the keys ascend with the lane index, at most
// `steps` of them.  True when sorted (then rank = lane).  The band arrives
// close to sorted -- the pool is ordered by its estimate -- so a few steps
// usually suffice.
__device__ __forceinline__ bool sort_lanes(unsigned long long& k, int lane, int steps) {
    for (int st = 0; st <= steps; ++st) {
        const unsigned long long prev = __shfl_up_sync(0xffffffffu, k, 1);
        if (__all_sync(0xffffffffu, lane == 0 || prev <= k)) return true;
        if (st == steps) break;
        const int par = st & 1;
        const bool lower = ((lane - par) & 1) == 0;
        const int partner = lower ? lane + 1 : lane - 1;
        const bool valid = partner >= 0 && partner < 32;
        const unsigned long long o = __shfl_sync(0xffffffffu, k, valid ? partner : lane);
        if (valid) k = lower ? (o < k ? o : k) : (o > k ? o : k);
    }
    return false;
}

// Final selection: members carry key (float(d32) bits << 32 | offset);
// non-members carry kNone.  FP64 refinement at the K-th boundary, then write
// ranks < K (and the padding).
template <int S, class Src, class T>
__device__ void select_and_write(const RerankParams& P, const RerankJob& J, const Src& X,
                                 const T* ref, const unsigned long long (&key_in)[S], int nb,
                                 int lane, size_t r) {
    unsigned long long key[S];
#pragma unroll
    for (int i = 0; i < S; ++i) key[i] = key_in[i];
    int rank[S];
    bool ranked = false;
    if constexpr (S == 1) {
        ranked = sort_lanes(key[0], lane, 6);
        rank[0] = lane;
    }
    if (!ranked) warp_rank(key, rank);
    double d64[S];
    bool refined[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
        refined[i] = false;
        d64[i] = 0.0;
    }
    if (nb > P.K) {
        unsigned din_b = 0u, dout_b = 0u;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const unsigned db = (unsigned)(key[i] >> 32);
            if (rank[i] == P.K - 1) din_b = db;
            if (rank[i] == P.K) dout_b = db;
        }
        // distances are non-negative: their bits order as unsigned integers
        const float din = __uint_as_float(__reduce_max_sync(0xffffffffu, din_b));
        const float dout = __uint_as_float(__reduce_max_sync(0xffffffffu, dout_b));
        const float tol = P.gamma * (din + dout);
        if (dout - din <= tol) {
            // boundary members: FP64 distances decide their order
            int nrec = 0;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const float d = __uint_as_float((unsigned)(key[i] >> 32));
                if (key[i] != kNone && d >= din - 2.f * tol && d <= dout + 2.f * tol) {
                    const int off = (int)(unsigned)(key[i] & 0xffffffffu);
                    const int yc = fast_div(off, J.wdiv);
                    d64[i] = direct_f64(X, P.p, P.C, ref, yc, off - yc * J.W);
                    refined[i] = true;
                    ++nrec;
                }
            }
            nrec = (int)__reduce_add_sync(0xffffffffu, (unsigned)nrec);
            if (lane == 0 && nrec) atomicAdd(P.counters + 1, (unsigned long long)nrec);
            // The refined members occupy a contiguous range of ranks (they are
            // exactly the members whose FP32 distance lies in the boundary
            // interval); re-rank them among themselves by (FP64 distance, offset).
            int start = INT_MAX;
#pragma unroll
            for (int i = 0; i < S; ++i)
                if (refined[i]) start = min(start, rank[i]);
            start = __reduce_min_sync(0xffffffffu, start);
            int sub[S];
#pragma unroll
            for (int i = 0; i < S; ++i) sub[i] = 0;
#pragma unroll
            for (int slot = 0; slot < S; ++slot) {
                for (int src = 0; src < 32; ++src) {
                    const int rm = __shfl_sync(0xffffffffu, refined[slot] ? 1 : 0, src);
                    const double dm = __shfl_sync(0xffffffffu, d64[slot], src);
                    const unsigned long long km = __shfl_sync(0xffffffffu, key[slot], src);
                    if (!rm) continue;
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        const bool before =
                            dm < d64[i] ||
                            (dm == d64[i] && (km & 0xffffffffull) < (key[i] & 0xffffffffull));
                        sub[i] += (refined[i] && before) ? 1 : 0;
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < S; ++i)
                if (refined[i]) rank[i] = start + sub[i];
        }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
        if (key[i] != kNone && rank[i] < P.K) {
            J.out_idx[r * P.K + rank[i]] = (int32_t)(unsigned)(key[i] & 0xffffffffu);
            J.out_dist[r * P.K + rank[i]] =
                refined[i] ? (float)d64[i] : __uint_as_float((unsigned)(key[i] >> 32));
        }
    }
    for (int k = nb + lane; k < P.K; k += 32) {
        J.out_idx[r * P.K + k] = -1;
        J.out_dist[r * P.K + k] = __int_as_float(0x7f800000);
    }
}

// The warp's pool entries of one reference (slot i holds entry lane + 32 i).
template <int S>
struct PoolRegs {
    int off[S];
    float v[S];
    __device__ __forceinline__ void load(const RerankParams& P, const RerankJob& J, size_t r, int lane) {
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const int k = lane + 32 * i;
            off[i] = -1;
            v[i] = 0.f;
            if (k < P.L) {
                off[i] = __ldg(J.pool_idx + r * P.L + k);
                v[i] = __ldg(J.pool_score + r * P.L + k);
            }
        }
    }
};

// Steps 1, 2 and 4 of the file header for reference (ry, rx) of job J, and
// step 3 with the output unless the band overflows.  X holds every pixel of
// the patches of its window, N (C = 1) every norm of its window.  Returns
// true on overflow: nothing is written and U is the (K+1)-th smallest key of
// the pool's direct distances (the window is recomputed).
template <int S, class Src, class T, int FP = 0, int FC = 0>
__device__ bool rerank_ref(const RerankParams& P, const RerankJob& J, const Src& X, const PlainSrc& N,
                           int ry, int rx, int lane, const PoolRegs<S>& pool, unsigned long long& U) {
    const size_t r = (size_t)ry * J.n_rx + rx;
    const int yr = ry * P.s, xr = rx * P.s;
    const T* ref = X.at(yr, xr);  // reference rows at ref + u * X.pitch
    const float nr = *N.at(yr, xr);

    // ---- the pool (best first; empty slots have offset -1)
    float v[S], nc[S];
    int yc[S], xc[S];
    int npool = 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const int off = pool.off[i];
        v[i] = -__int_as_float(0x7f800000);
        nc[i] = 0.f;
        yc[i] = 0;
        xc[i] = 0;
        if (off >= 0) {
            yc[i] = fast_div(off, J.wdiv);
            xc[i] = off - yc[i] * J.W;
            v[i] = pool.v[i];
            nc[i] = *N.at(yc[i], xc[i]);
        }
        npool += __popc(__ballot_sync(0xffffffffu, off >= 0));
    }

    // ---- band: entries with v >= tb (see the file header); the pool is
    // sorted, so the K-th largest score is entry K-1
    bool member[S];
#pragma unroll
    for (int i = 0; i < S; ++i) member[i] = pool.off[i] >= 0;
    int nb = npool;
    bool overflow = false;
    if (npool > P.K) {
        float vK = 0.f;
        unsigned ncmax = 0u, vabs = 0u;  // bits of non-negative floats order as integers
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const int k = lane + 32 * i;
            const float vs = __shfl_sync(0xffffffffu, v[i], (P.K - 1) & 31);
            if (i == (P.K - 1) >> 5) vK = vs;
            if (k < P.K) {
                ncmax = max(ncmax, __float_as_uint(nc[i]));
                vabs = max(vabs, __float_as_uint(fabsf(v[i])));
            }
        }
        const float ncm = __uint_as_float(__reduce_max_sync(0xffffffffu, ncmax));
        const float va = __uint_as_float(__reduce_max_sync(0xffffffffu, vabs));
        const float tb = vK - P.round_rel * va * 1.001f - 2.0f * kEps * (nr + ncm) * 1.0001f;
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            member[i] = pool.off[i] >= 0 && v[i] >= tb;
            cnt += __popc(__ballot_sync(0xffffffffu, member[i]));
        }
        nb = cnt;
        overflow = (npool == P.L) && (nb == P.L);
    }

    unsigned long long key[S];
    int viol = 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        key[i] = kNone;
        if (member[i]) {
            float d32;
            if constexpr (!std::is_same<Src, PlainSrc>::value)
                d32 = direct_f32<FP, FC>(X, P.p, P.C, ref, yc[i], xc[i]);
            else
                d32 = direct_f32(X, P.p, P.C, ref, yc[i], xc[i]);
            key[i] = ((unsigned long long)__float_as_uint(d32) << 32) | (unsigned)pool.off[i];
            // identity estimate d~ = n_r - 2 (v - eps n_j) against its bound 2 eps (n_r + n_j)
            const float dt = nr - 2.0f * (v[i] - kEps * nc[i]);
            if (fabsf(dt - d32) > 2.0f * kEps * (nr + nc[i]) + 2.0f * P.round_rel * fabsf(v[i]) +
                                      P.gamma * d32 + 1e-6f * (nr + nc[i]) + 1.0f)
                ++viol;
        }
    }
    viol = (int)__reduce_add_sync(0xffffffffu, (unsigned)viol);
    if (lane == 0 && viol) atomicAdd(P.counters + 2, (unsigned long long)viol);
    if (overflow) {
        // every entry is a member (L > K): the key of rank K exists and is unique
        int rank[S];
        warp_rank(key, rank);
        U = kNone;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const unsigned b = __ballot_sync(0xffffffffu, rank[i] == P.K);
            if (b) U = __shfl_sync(0xffffffffu, key[i], __ffs(b) - 1);
        }
        return true;
    }
    select_and_write<S>(P, J, X, ref, key, nb, lane, r);
    return false;
}

// Inserts the warp's keys k (one per lane) into the sorted list of nl keys
// in shared memory (kNone-padded), keeping the nl smallest.
__device__ __forceinline__ void list_insert(unsigned long long k, unsigned long long* list, int nl,
                                            int lane) {
    unsigned pass = __ballot_sync(0xffffffffu, k < list[nl - 1]);
    while (pass) {
        const int src = __ffs(pass) - 1;
        pass &= pass - 1;
        const unsigned long long kk = __shfl_sync(0xffffffffu, k, src);
        if (!(kk < list[nl - 1])) continue;
        int pos = 0;
        for (int e = lane; e < nl; e += 32) pos += list[e] < kk ? 1 : 0;
        pos = (int)__reduce_add_sync(0xffffffffu, (unsigned)pos);
        unsigned long long nv[kFbSlots];
#pragma unroll
        for (int t = 0; t < kFbSlots; ++t) {
            const int e = lane + 32 * t;
            nv[t] = e < nl ? (e > pos ? list[e - 1] : (e == pos ? kk : list[e])) : kNone;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kFbSlots; ++t)
            if (lane + 32 * t < nl) list[lane + 32 * t] = nv[t];
        __syncwarp();
    }
}

// Overflow, share `part` of `nparts`: the exact top-(K+1) of the window
// candidates 32 part + lane + 32 nparts m (FP32 direct distances) into list.
template <class Src, class T>
__device__ void window_part(const RerankParams& P, const RerankJob& J, const Src& X, int ry, int rx,
                            int part, int nparts, int lane, unsigned long long* list) {
    const int nl = P.K + 1;
    const int yr = ry * P.s, xr = rx * P.s;
    const T* ref = X.at(yr, xr);
    for (int e = lane; e < kFbSlots * 32; e += 32) list[e] = kNone;
    __syncwarp();
    const int y0 = max(0, yr - P.h), y1 = min(J.Hc - 1, yr + P.h);
    const int x0 = max(0, xr - P.h), x1 = min(J.Wc - 1, xr + P.h);
    const int nxw = x1 - x0 + 1;
    const int total = (y1 - y0 + 1) * nxw;
    for (int base = part * 32; base < total; base += 32 * nparts) {
        const int i = base + lane;
        unsigned long long k = kNone;
        if (i < total) {
            const int yc = y0 + i / nxw, xc = x0 + i % nxw;
            const float d = direct_f32(X, P.p, P.C, ref, yc, xc);
            k = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(yc * J.W + xc);
        }
        list_insert(k, list, nl, lane);
    }
}

// Overflow, share `part` of `nparts` of the window (candidates
// 32 part + lane + 32 nparts m): FP32 direct-distance keys <= U appended to
// cand (slots past kCandCap are counted but not stored).
template <class Src, class T>
__device__ void window_filter(const RerankParams& P, const RerankJob& J, const Src& X, int ry, int rx,
                              int part, int nparts, int lane, unsigned long long U,
                              unsigned long long* cand, int* cand_n) {
    const int yr = ry * P.s, xr = rx * P.s;
    const T* ref = X.at(yr, xr);
    const int y0 = max(0, yr - P.h), y1 = min(J.Hc - 1, yr + P.h);
    const int x0 = max(0, xr - P.h), x1 = min(J.Wc - 1, xr + P.h);
    const int nxw = x1 - x0 + 1;
    const int total = (y1 - y0 + 1) * nxw;
    for (int i = part * 32 + lane; i < total; i += 32 * nparts) {
        const int yc = y0 + i / nxw, xc = x0 + i % nxw;
        const float d = direct_f32(X, P.p, P.C, ref, yc, xc);
        const unsigned long long k = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(yc * J.W + xc);
        if (k <= U) {
            const int slot = atomicAdd(cand_n, 1);
            if (slot < kCandCap) cand[slot] = k;
        }
    }
}

// The list's keys through select_and_write.
template <class Src, class T>
__device__ void write_list(const RerankParams& P, const RerankJob& J, const Src& X, int ry, int rx,
                           int lane, const unsigned long long* list) {
    const int nl = P.K + 1;
    unsigned long long key2[kFbSlots];
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < kFbSlots; ++t) {
        const int e = lane + 32 * t;
        key2[t] = e < nl ? list[e] : kNone;
        cnt += __popc(__ballot_sync(0xffffffffu, key2[t] != kNone));
    }
    const T* ref = X.at(ry * P.s, rx * P.s);
    select_and_write<kFbSlots>(P, J, X, ref, key2, cnt, lane, (size_t)ry * J.n_rx + rx);
}

// Tile t of the launch: its job (binary search over the jobs' first tiles).
__device__ __forceinline__ int tile_job(const RerankParams& P, int t) {
    int lo = 0, hi = P.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.jobs[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// FP, FC: patch side and channels fixed at compile time (0: from P).
// kQuad: the region stored plainly (C a multiple of 4), else as element pairs.
// NW: warps per block (16 where the region leaves room for at most two blocks per SM).
template <int S, int FP, int FC, bool kQuad, int NW = kTileWarps>
__global__ void __launch_bounds__(NW * 32) rerank_tile_kernel(const __grid_constant__ RerankParams P) {
    using Src = typename std::conditional<kQuad, QuadSrc, PairSrc>::type;
    using T = typename std::conditional<kQuad, float, float2>::type;
    extern __shared__ __align__(16) float2 sm2[];
    __shared__ unsigned long long list_s[kFbSlots * 32];  // overflow: window keys, then a list
    __shared__ unsigned long long ovf_u[kMaxTileRefs];
    __shared__ int ovf_ref[kMaxTileRefs];
    __shared__ int ovf_n, cand_n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x;
    const RerankJob& J = P.jobs[tile_job(P, t)];
    const int lt = t - J.tile_begin;
    const int ry0 = (lt / J.tiles_x) * P.TRY, rx0 = (lt % J.tiles_x) * P.TRX;
    const int ry1 = min(ry0 + P.TRY, J.n_ry) - 1, rx1 = min(rx0 + P.TRX, J.n_rx) - 1;
    const int ncols = rx1 - rx0 + 1;
    const int nref = (ry1 - ry0 + 1) * ncols;
    // the warp's first pool, in flight while the region is staged
    PoolRegs<S> pool;
    if (warp < nref) pool.load(P, J, (size_t)(ry0 + warp / ncols) * J.n_rx + rx0 + warp % ncols, lane);
    if (threadIdx.x == 0) ovf_n = 0;
    // region: every pixel of every window patch of the tile's references
    const int iy0 = max(0, ry0 * P.s - P.h), iy1 = min(J.H - 1, ry1 * P.s + P.h + P.p - 1);
    const int ix0 = max(0, rx0 * P.s - P.h), ix1 = min(J.W - 1, rx1 * P.s + P.h + P.p - 1);
    const int ny1 = min(J.Hc - 1, ry1 * P.s + P.h), nx1 = min(J.Wc - 1, rx1 * P.s + P.h);
    const int ipitch = (ix1 - ix0 + 1) * P.C, npitch = nx1 - ix0 + 1;
    float2* simg = sm2;
    float* snrm = reinterpret_cast<float*>(sm2 + P.img_cap);
    const int irows = iy1 - iy0 + 1, nrows = ny1 - iy0 + 1;
    for (int y = warp; y < irows; y += NW) {
        const float* g = J.img + ((size_t)(iy0 + y) * J.W + ix0) * P.C;
        if constexpr (kQuad) {
            float* row = reinterpret_cast<float*>(sm2) + y * ipitch;
            for (int e = lane; e < ipitch; e += 32) row[e] = __ldg(g + e);
        } else {
            for (int e0 = 0; e0 < ipitch; e0 += 32) {
                const int e = e0 + lane;
                const float a = e < ipitch ? __ldg(g + e) : 0.f;
                float b = __shfl_down_sync(0xffffffffu, a, 1);
                if (lane == 31) b = e + 1 < ipitch ? __ldg(g + e + 1) : 0.f;
                if (e < ipitch) simg[y * ipitch + e] = make_float2(a, b);
            }
        }
    }
    for (int y = warp; y < nrows; y += NW) {
        const float* g = J.nrm + (size_t)(iy0 + y) * J.Wc + ix0;
        for (int x = lane; x < npitch; x += 32) snrm[y * npitch + x] = __ldg(g + x);
    }
    __syncthreads();
    const Src X{reinterpret_cast<const T*>(sm2), iy0, ix0, ipitch, P.C};
    const PlainSrc N{snrm, iy0, ix0, npitch, 1};
    // references i = warp + 8 m, row-major in the tile: (qi, ri) = divmod(i, ncols)
    int qi = warp / ncols, ri = warp % ncols;
    for (int i = warp; i < nref; i += NW) {
        const PoolRegs<S> cur = pool;
        const int ry = ry0 + qi, rx = rx0 + ri;
        ri += NW;
        while (ri >= ncols) {
            ri -= ncols;
            ++qi;
        }
        if (i + NW < nref) pool.load(P, J, (size_t)(ry0 + qi) * J.n_rx + rx0 + ri, lane);
        unsigned long long U;
        if (rerank_ref<S, Src, T, FP, FC>(P, J, X, N, ry, rx, lane, cur, U) && lane == 0) {
            const int o = atomicAdd(&ovf_n, 1);
            ovf_ref[o] = i;
            ovf_u[o] = U;
        }
    }
    __syncthreads();
    // overflow references: every warp filters a share of the window by U
    const int novf = ovf_n;
    for (int o = 0; o < novf; ++o) {
        const int i = ovf_ref[o];
        const int ry = ry0 + i / ncols, rx = rx0 + i % ncols;
        if (threadIdx.x == 0) {
            cand_n = 0;
            atomicAdd(P.counters + 0, 1ull);
        }
        __syncthreads();
        window_filter<Src, T>(P, J, X, ry, rx, warp, NW, lane, ovf_u[o], list_s, &cand_n);
        __syncthreads();
        const int n = cand_n;
        if (warp == 0) {
            if (n <= kCandCap) {
                unsigned long long key[kFbSlots];
#pragma unroll
                for (int t = 0; t < kFbSlots; ++t)
                    key[t] = lane + 32 * t < n ? list_s[lane + 32 * t] : kNone;
                __syncwarp();
                select_and_write<kFbSlots>(P, J, X, X.at(ry * P.s, rx * P.s), key, n, lane,
                                           (size_t)ry * J.n_rx + rx);
            } else {
                // more ties than the buffer holds: the exact top-(K+1) by insertion
                window_part<Src, T>(P, J, X, ry, rx, 0, 1, lane, list_s);
                write_list<Src, T>(P, J, X, ry, rx, lane, list_s);
            }
        }
        __syncthreads();
    }
}

// The same steps on global memory: one image, one reference per warp.
template <int S>
__global__ void __launch_bounds__(128) rerank_global_kernel(const __grid_constant__ RerankParams P) {
    __shared__ unsigned long long list_s[4][kFbSlots * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RerankJob& J = P.jobs[0];
    const size_t r = (size_t)blockIdx.x * 4 + warp;
    if (r >= (size_t)J.n_ry * J.n_rx) return;
    const PlainSrc X{J.img, 0, 0, J.W * P.C, P.C};
    const PlainSrc N{J.nrm, 0, 0, J.Wc, 1};
    const int ry = (int)(r / J.n_rx), rx = (int)(r % J.n_rx);
    PoolRegs<S> pool;
    pool.load(P, J, r, lane);
    unsigned long long U;
    if (rerank_ref<S, PlainSrc, float>(P, J, X, N, ry, rx, lane, pool, U)) {
        if (lane == 0) atomicAdd(P.counters + 0, 1ull);
        window_part<PlainSrc, float>(P, J, X, ry, rx, 0, 1, lane, list_s[warp]);
        write_list<PlainSrc, float>(P, J, X, ry, rx, lane, list_s[warp]);
    }
}

// Region layout: plain (16-byte patch rows) when C is a multiple of 4.
bool quad_layout(const Geom& g) { return g.C % 4 == 0; }

// Tile shape and shared memory for a class; false: no region fits.
bool tile_shape(const Geom& g, int& TRY, int& TRX, int& img_cap, int& smem) {
    static const int kShapes[5][2] = {{8, 8}, {4, 8}, {4, 4}, {2, 2}, {1, 1}};
    for (const auto& sh : kShapes) {
        const int rows = (sh[0] - 1) * g.s + 2 * g.h + g.p;
        const int cols = (sh[1] - 1) * g.s + 2 * g.h + g.p;
        // capacity in 8-byte units: element pairs, or two plain elements
        img_cap = quad_layout(g) ? (rows * cols * g.C + 1) / 2 : (rows * cols * g.C + 1) / 2 * 2;
        smem = img_cap * 8 + (rows - g.p + 1) * (cols - g.p + 1) * 4;
        if (smem <= kTileSmemLimit) {
            TRY = sh[0];
            TRX = sh[1];
            return true;
        }
    }
    return false;
}

template <int S>
cudaError_t launch_s(const RerankParams& P, bool tiled, int smem, int grid, cudaStream_t st) {
    void (*kern)(RerankParams) = nullptr;
    // four-channel regions over a quarter of the shared memory fit at most two
    // blocks per SM: those blocks take 16 warps instead of 8 (pools up to 96)
    constexpr int S3 = S <= 3 ? S : 1;
    const bool wide = tiled && P.C % 4 == 0 && S <= 3 && smem > kTileSmemLimit / 4;
    if (tiled && P.p == 8 && P.C == 1) kern = rerank_tile_kernel<S, 8, 1, false>;  // 8 x 8 grey, unrolled
    else if (wide && P.p == 8 && P.C == 4) kern = rerank_tile_kernel<S3, 8, 4, true, 16>;
    else if (wide) kern = rerank_tile_kernel<S3, 0, 0, true, 16>;
    else if (tiled && P.p == 8 && P.C == 4 && S <= 3) kern = rerank_tile_kernel<S3, 8, 4, true>;
    else if (tiled && P.C % 4 == 0) kern = rerank_tile_kernel<S, 0, 0, true>;
    else if (tiled) kern = rerank_tile_kernel<S, 0, 0, false>;
    if (kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kern<<<grid, (wide ? 16 : kTileWarps) * 32, smem, st>>>(P);
    } else {
        rerank_global_kernel<S><<<grid, 128, 0, st>>>(P);
    }
    return cudaGetLastError();
}

RerankJob make_job(const Geom& g, const RerankArgs& a) {
    RerankJob j{};
    j.img = a.img; j.nrm = a.nrm; j.pool_idx = a.pool_idx; j.pool_score = a.pool_score;
    j.out_idx = a.out_idx; j.out_dist = a.out_dist;
    j.H = g.H; j.W = g.W; j.n_ry = g.n_ry; j.n_rx = g.n_rx; j.Hc = g.Hc; j.Wc = g.Wc;
    j.wdiv = make_fastdiv((unsigned)g.W);
    return j;
}

}  // namespace

bool rerank_same_class(const Geom& a, const Geom& b) {
    return a.C == b.C && a.p == b.p && a.h == b.h && a.s == b.s && a.K == b.K && a.L == b.L &&
           tc_score_bits(a) == tc_score_bits(b);
}

cudaError_t launch_rerank_batch(const Geom* gs, const RerankArgs* as, int n,
                                unsigned long long* counters, cudaStream_t st, int* nlaunch) {
    if (nlaunch) *nlaunch = 0;
    int i = 0;
    while (i < n) {
        static thread_local RerankParams P;
        P = RerankParams{};
        const Geom& g = gs[i];
        P.C = g.C; P.p = g.p; P.h = g.h; P.s = g.s; P.K = g.K; P.L = g.L;
        const int tb = tc_score_bits(g);
        P.round_rel = tb ? ldexpf(1.0f, tb - 23) : 0.0f;
        P.gamma = (float)(g.p * g.p * g.C + 3) * 5.9604645e-08f;  // (n + 3) 2^-24
        P.counters = counters;
        const int S = (g.L + 31) / 32;
        if (S < 1 || S > 5) return cudaErrorNotSupported;
        int smem = 0;
        const bool tiled = tile_shape(g, P.TRY, P.TRX, P.img_cap, smem);
        int nj = 0, tiles = 0, grid;
        if (tiled) {
            while (i < n && nj < kMaxRerankJobs && rerank_same_class(gs[i], g)) {
                RerankJob& j = P.jobs[nj];
                j = make_job(gs[i], as[i]);
                j.tiles_x = (gs[i].n_rx + P.TRX - 1) / P.TRX;
                j.tile_begin = tiles;
                tiles += j.tiles_x * ((gs[i].n_ry + P.TRY - 1) / P.TRY);
                ++nj;
                ++i;
            }
            grid = tiles;
        } else {
            P.jobs[0] = make_job(gs[i], as[i]);
            nj = 1;
            ++i;
            grid = (g.nR + 3) / 4;
        }
        P.njobs = nj;
        P.total_tiles = tiles;
        cudaError_t e;
        switch (S) {
            case 1: e = launch_s<1>(P, tiled, smem, grid, st); break;
            case 2: e = launch_s<2>(P, tiled, smem, grid, st); break;
            case 3: e = launch_s<3>(P, tiled, smem, grid, st); break;
            case 4: e = launch_s<4>(P, tiled, smem, grid, st); break;
            default: e = launch_s<5>(P, tiled, smem, grid, st); break;
        }
        if (e != cudaSuccess) return e;
        if (nlaunch) ++*nlaunch;
    }
    return cudaSuccess;
}

cudaError_t launch_rerank(const Geom& g, const float* img, const float* nrm,
                          const int32_t* pool_idx, const float* pool_score, int32_t* out_idx,
                          float* out_dist, unsigned long long* counters, cudaStream_t st) {
    const RerankArgs a{img, nrm, pool_idx, pool_score, out_idx, out_dist};
    return launch_rerank_batch(&g, &a, 1, counters, st);
}

}  // namespace bm
