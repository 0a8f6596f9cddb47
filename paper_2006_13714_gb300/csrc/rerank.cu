// rerank.cu -- (a6) float32 boundary re-rank.
//
// The tensor-core pass leaves, per reference r, a pool of the L largest
// v_j = b~_j + eps n_j (b~ the split-bf16 estimate of Theorem 1's score
// b_j = C_r(j) - 0.5 n_j of the centred patches, n_j = ||X_j - c||^2,
// eps = 2^-14), in any order.  The identity d = ||X_r||^2 - 2 b (Lemma 2)
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
// One warp per reference; every ranking uses 64-bit integer keys (FP64 is
// slow on this part and is kept to the rare boundary ties).
#include "bm_internal.h"

#include <climits>

namespace bm {
namespace {

constexpr float kEps = 6.103515625e-05f;  // 2^-14, same constant as the tensor-core pass
constexpr int kWarps = 4;
constexpr int kFbSlots = (kMaxK + 1 + 31) / 32;
constexpr unsigned long long kNone = ~0ull;

struct RerankParams {
    const float* img;
    const float* nrm;
    const int32_t* pool_idx;
    const float* pool_score;
    int32_t* out_idx;
    float* out_dist;
    unsigned long long* counters;  // [0] overflow, [1] fp64 rechecks, [2] bound violations
    int H, W, C, p, h, s, K, L, n_ry, n_rx, Wc, nR;
    float round_rel;  // pool-score rounding, relative: 2^(tbits - 23) (0: exact scores)
};

__device__ __forceinline__ float direct_f32(const RerankParams& P, const float* ref, int yc, int xc) {
    const int pc = P.p * P.C;
    float acc = 0.f;
    for (int u = 0; u < P.p; ++u) {
        const float* crow = P.img + ((size_t)(yc + u) * P.W + xc) * P.C;
        const float* rrow = ref + u * pc;
#pragma unroll 8
        for (int e = 0; e < pc; ++e) {
            const float d = rrow[e] - __ldg(crow + e);
            acc = fmaf(d, d, acc);
        }
    }
    return acc;
}

__device__ __forceinline__ double direct_f64(const RerankParams& P, const float* ref, int yc, int xc) {
    const int pc = P.p * P.C;
    double acc = 0.0;
    for (int u = 0; u < P.p; ++u) {
        const float* crow = P.img + ((size_t)(yc + u) * P.W + xc) * P.C;
        const float* rrow = ref + u * pc;
        for (int e = 0; e < pc; ++e) {
            const double d = (double)rrow[e] - (double)__ldg(crow + e);
            acc = fma(d, d, acc);
        }
    }
    return acc;
}

// rank[i] = number of keys (over all 32*S lane-strided slots) smaller than key[i].
template <int S>
__device__ __forceinline__ void warp_rank(const unsigned long long (&key)[S], int (&rank)[S]) {
#pragma unroll
    for (int i = 0; i < S; ++i) rank[i] = 0;
#pragma unroll
    for (int slot = 0; slot < S; ++slot) {
        for (int src = 0; src < 32; ++src) {
            const unsigned long long km = __shfl_sync(0xffffffffu, key[slot], src);
#pragma unroll
            for (int i = 0; i < S; ++i) rank[i] += km < key[i] ? 1 : 0;
        }
    }
}

__device__ __forceinline__ unsigned orderable(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Final selection: members carry key (float(d32) bits << 32 | offset);
// non-members carry kNone.  FP64 refinement at the K-th boundary, then write
// ranks < K (and the padding).
template <int S>
__device__ void select_and_write(const RerankParams& P, const float* ref,
                                 const unsigned long long (&key)[S], int nb, int lane, size_t r,
                                 float gamma) {
    int rank[S];
    warp_rank(key, rank);
    double d64[S];
    bool refined[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
        refined[i] = false;
        d64[i] = 0.0;
    }
    if (nb > P.K) {
        float din = 0.f, dout = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const float d = __uint_as_float((unsigned)(key[i] >> 32));
            if (rank[i] == P.K - 1) din = d;
            if (rank[i] == P.K) dout = d;
        }
        for (int o = 16; o > 0; o >>= 1) {
            din = fmaxf(din, __shfl_xor_sync(0xffffffffu, din, o));
            dout = fmaxf(dout, __shfl_xor_sync(0xffffffffu, dout, o));
        }
        const float tol = gamma * (din + dout);
        if (dout - din <= tol) {
            // boundary members: FP64 distances decide their order
            int nrec = 0;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const float d = __uint_as_float((unsigned)(key[i] >> 32));
                if (key[i] != kNone && d >= din - 2.f * tol && d <= dout + 2.f * tol) {
                    const int off = (int)(unsigned)(key[i] & 0xffffffffu);
                    d64[i] = direct_f64(P, ref, off / P.W, off % P.W);
                    refined[i] = true;
                    ++nrec;
                }
            }
            for (int o = 16; o > 0; o >>= 1) nrec += __shfl_xor_sync(0xffffffffu, nrec, o);
            if (lane == 0 && nrec) atomicAdd(P.counters + 1, (unsigned long long)nrec);
            // The refined members occupy a contiguous range of ranks (they are
            // exactly the members whose FP32 distance lies in the boundary
            // interval); re-rank them among themselves by (FP64 distance, offset).
            int start = INT_MAX;
#pragma unroll
            for (int i = 0; i < S; ++i)
                if (refined[i]) start = min(start, rank[i]);
            for (int o = 16; o > 0; o >>= 1) start = min(start, __shfl_xor_sync(0xffffffffu, start, o));
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
            P.out_idx[r * P.K + rank[i]] = (int32_t)(unsigned)(key[i] & 0xffffffffu);
            P.out_dist[r * P.K + rank[i]] =
                refined[i] ? (float)d64[i] : __uint_as_float((unsigned)(key[i] >> 32));
        }
    }
    for (int k = nb + lane; k < P.K; k += 32) {
        P.out_idx[r * P.K + k] = -1;
        P.out_dist[r * P.K + k] = __int_as_float(0x7f800000);
    }
}

template <int S>
__global__ void __launch_bounds__(kWarps * 32) rerank_kernel(const __grid_constant__ RerankParams P) {
    __shared__ float ref_s[kWarps][kMaxPatchElems];
    __shared__ unsigned long long list_s[kWarps][kFbSlots * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t r = (size_t)blockIdx.x * kWarps + warp;
    if (r >= (size_t)P.nR) return;
    const int ry = (int)(r / P.n_rx), rx = (int)(r % P.n_rx);
    const int yr = ry * P.s, xr = rx * P.s;
    const int pc = P.p * P.C;
    for (int e = lane; e < P.p * pc; e += 32) {
        const int u = e / pc, k = e % pc;
        ref_s[warp][e] = P.img[((size_t)(yr + u) * P.W + xr) * P.C + k];
    }
    __syncwarp();
    const float* ref = ref_s[warp];
    const float nr = P.nrm[(size_t)yr * P.Wc + xr];
    const float gamma = (float)(pc * P.p + 3) * 5.9604645e-08f;  // (n + 3) 2^-24

    // ---- load the pool (any order; empty slots have offset -1)
    float v[S], nc[S];
    int off[S];
    int npool = 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const int k = lane + 32 * i;
        v[i] = -__int_as_float(0x7f800000);
        off[i] = -1;
        nc[i] = 0.f;
        if (k < P.L) {
            off[i] = P.pool_idx[r * P.L + k];
            if (off[i] >= 0) {
                v[i] = P.pool_score[r * P.L + k];
                nc[i] = P.nrm[(size_t)(off[i] / P.W) * P.Wc + (off[i] % P.W)];
                ++npool;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) npool += __shfl_xor_sync(0xffffffffu, npool, o);

    // ---- band: entries with v >= T' (see the file header)
    bool member[S];
#pragma unroll
    for (int i = 0; i < S; ++i) member[i] = off[i] >= 0;
    int nb = npool;
    bool overflow = false;
    if (npool > P.K) {
        // rank by v descending (ties: slot index)
        unsigned long long vk[S];
#pragma unroll
        for (int i = 0; i < S; ++i)
            vk[i] = ((unsigned long long)(~orderable(v[i])) << 32) | (unsigned)(lane + 32 * i);
        int rk[S];
        warp_rank(vk, rk);
        float vK = -__int_as_float(0x7f800000), ncmax = 0.f, vabs = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            if (off[i] >= 0 && rk[i] == P.K - 1) vK = v[i];
            if (off[i] >= 0 && rk[i] < P.K) {
                ncmax = fmaxf(ncmax, nc[i]);
                vabs = fmaxf(vabs, fabsf(v[i]));
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            vK = fmaxf(vK, __shfl_xor_sync(0xffffffffu, vK, o));
            ncmax = fmaxf(ncmax, __shfl_xor_sync(0xffffffffu, ncmax, o));
            vabs = fmaxf(vabs, __shfl_xor_sync(0xffffffffu, vabs, o));
        }
        const float tb = vK - P.round_rel * vabs * 1.001f - 2.0f * kEps * (nr + ncmax) * 1.0001f;
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            member[i] = off[i] >= 0 && v[i] >= tb;
            cnt += member[i] ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        nb = cnt;
        overflow = (npool == P.L) && (nb == P.L);
    }

    if (!overflow) {
        unsigned long long key[S];
        int viol = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            key[i] = kNone;
            if (member[i]) {
                const float d32 = direct_f32(P, ref, off[i] / P.W, off[i] % P.W);
                key[i] = ((unsigned long long)__float_as_uint(d32) << 32) | (unsigned)off[i];
                // identity estimate d~ = n_r - 2 (v - eps n_j) against its bound 2 eps (n_r + n_j)
                const float dt = nr - 2.0f * (v[i] - kEps * nc[i]);
                if (fabsf(dt - d32) > 2.0f * kEps * (nr + nc[i]) + 2.0f * P.round_rel * fabsf(v[i]) +
                                          gamma * d32 + 1e-6f * (nr + nc[i]) + 1.0f)
                    ++viol;
            }
        }
        for (int o = 16; o > 0; o >>= 1) viol += __shfl_xor_sync(0xffffffffu, viol, o);
        if (lane == 0 && viol) atomicAdd(P.counters + 2, (unsigned long long)viol);
        select_and_write<S>(P, ref, key, nb, lane, r, gamma);
        return;
    }

    // ---- overflow: exact top-(K+1) over the whole window, FP32 direct distances
    if (lane == 0) atomicAdd(P.counters + 0, 1ull);
    unsigned long long* list = list_s[warp];
    const int nl = P.K + 1;
    for (int e = lane; e < kFbSlots * 32; e += 32) list[e] = kNone;
    __syncwarp();
    const int Hc = P.H - P.p + 1;
    const int y0 = max(0, yr - P.h), y1 = min(Hc - 1, yr + P.h);
    const int x0 = max(0, xr - P.h), x1 = min(P.Wc - 1, xr + P.h);
    const int nxw = x1 - x0 + 1;
    const int total = (y1 - y0 + 1) * nxw;
    for (int base = 0; base < total; base += 32) {
        const int i = base + lane;
        unsigned long long k = kNone;
        if (i < total) {
            const int yc = y0 + i / nxw, xc = x0 + i % nxw;
            const float d = direct_f32(P, ref, yc, xc);
            k = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(yc * P.W + xc);
        }
        unsigned pass = __ballot_sync(0xffffffffu, k < list[nl - 1]);
        while (pass) {
            const int src = __ffs(pass) - 1;
            pass &= pass - 1;
            const unsigned long long kk = __shfl_sync(0xffffffffu, k, src);
            if (!(kk < list[nl - 1])) continue;
            int pos = 0;
            for (int e = lane; e < nl; e += 32) pos += list[e] < kk ? 1 : 0;
            for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
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
    unsigned long long key2[kFbSlots];
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < kFbSlots; ++t) {
        const int e = lane + 32 * t;
        key2[t] = e < nl ? list[e] : kNone;
        cnt += key2[t] != kNone ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    select_and_write<kFbSlots>(P, ref, key2, cnt, lane, r, gamma);
}

}  // namespace

cudaError_t launch_rerank(const Geom& g, const float* img, const float* nrm,
                          const int32_t* pool_idx, const float* pool_score, int32_t* out_idx,
                          float* out_dist, unsigned long long* counters, cudaStream_t st) {
    RerankParams P{};
    P.img = img; P.nrm = nrm; P.pool_idx = pool_idx; P.pool_score = pool_score;
    P.out_idx = out_idx; P.out_dist = out_dist; P.counters = counters;
    P.H = g.H; P.W = g.W; P.C = g.C; P.p = g.p; P.h = g.h; P.s = g.s; P.K = g.K; P.L = g.L;
    P.n_ry = g.n_ry; P.n_rx = g.n_rx; P.Wc = g.Wc; P.nR = g.nR;
    const int tb = tc_score_bits(g);
    P.round_rel = tb ? ldexpf(1.0f, tb - 23) : 0.0f;
    const int blocks = (g.nR + kWarps - 1) / kWarps;
    switch ((g.L + 31) / 32) {
        case 1: rerank_kernel<1><<<blocks, kWarps * 32, 0, st>>>(P); break;
        case 2: rerank_kernel<2><<<blocks, kWarps * 32, 0, st>>>(P); break;
        case 3: rerank_kernel<3><<<blocks, kWarps * 32, 0, st>>>(P); break;
        case 4: rerank_kernel<4><<<blocks, kWarps * 32, 0, st>>>(P); break;
        case 5: rerank_kernel<5><<<blocks, kWarps * 32, 0, st>>>(P); break;
        default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace bm
