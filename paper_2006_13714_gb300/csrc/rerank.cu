// rerank.cu -- (a6) float32 boundary re-rank.
//
// The tensor-core pass leaves, per reference r, a pool of the L largest
// v_j = b~_j + eps n_j (b~ the split-bf16 estimate of Theorem 1's score
// b_j = C_r(j) - 0.5 n_j, n_j = ||X_j||^2, eps = 2^-14) sorted by v
// descending.  The identity d = ||X_r||^2 - 2 b (Lemma 2) loses precision to
// cancellation in proportion to ||X_r||^2 + ||X_j||^2, not to d, so the
// final distances are recomputed here directly:
//
//   1. Error bound: |b~_j - b_j| <= eps (n_r + n_j).  At least K pool
//      entries have b >= T' = v_K - eps n_r - 2 eps max_{k<=K} n_k, so only
//      entries with u_j = v_j + eps n_r >= T' can be among the K nearest:
//      a prefix of the pool (the band).  If the pool is full and its last
//      entry is still in the band, candidates outside the pool might be too
//      ("overflow"): that reference is recomputed over its whole window.
//   2. Band members get the explicit FP32 distance sum (X_r - X_j)^2
//      (Eq. equ:bmMetric_app), relative error <= gamma = (n + 3) 2^-24 with
//      n = p*p*C terms, and are ranked by (distance, row-major offset).
//   3. If the K-th and (K+1)-th FP32 distances are within that error of each
//      other, the members near the boundary are recomputed in FP64 and the
//      order there is decided by the FP64 values.
//   4. Debug counter: band members whose identity estimate misses the direct
//      distance by more than the stated bound (should stay 0).
// One warp per reference.
#include "bm_internal.h"

#include <climits>

namespace bm {
namespace {

constexpr float kEps = 6.103515625e-05f;  // 2^-14, same constant as the tensor-core pass
constexpr int kWarps = 4;
constexpr int kMaxPool = 192;             // >= every pool length L
constexpr int kSlots = kMaxPool / 32;     // pool entries per lane
constexpr int kFbSlots = (kMaxK + 1 + 31) / 32;

struct RerankParams {
    const float* img;
    const float* nrm;
    const int32_t* pool_idx;
    const float* pool_score;
    int32_t* out_idx;
    float* out_dist;
    unsigned long long* counters;  // [0] overflow, [1] fp64 rechecks, [2] bound violations
    int H, W, C, p, h, s, K, L, n_ry, n_rx, Wc, nR;
};

__device__ __forceinline__ float direct_f32(const RerankParams& P, const float* ref, int yc, int xc) {
    const int pc = P.p * P.C;
    float acc = 0.f;
    for (int u = 0; u < P.p; ++u) {
        const float* crow = P.img + ((size_t)(yc + u) * P.W + xc) * P.C;
        const float* rrow = ref + u * pc;
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

template <int N>
__device__ __forceinline__ double pick(const double (&a)[N], int i) {
    double r = a[0];
#pragma unroll
    for (int k = 1; k < N; ++k) r = (i == k) ? a[k] : r;
    return r;
}
template <int N>
__device__ __forceinline__ int pick(const int (&a)[N], int i) {
    int r = a[0];
#pragma unroll
    for (int k = 1; k < N; ++k) r = (i == k) ? a[k] : r;
    return r;
}

// Rank of every member (lane-strided slots) by (key, off) ascending.
template <int N>
__device__ void rank_members(const double (&key)[N], const int (&off)[N], int nslots, int lane,
                             int (&rank)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) rank[i] = 0;
    for (int m = 0; m < nslots; ++m) {
        const int src = m & 31, slot = m >> 5;
        const double km = __shfl_sync(0xffffffffu, pick(key, slot), src);
        const int om = __shfl_sync(0xffffffffu, pick(off, slot), src);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const bool lt = km < key[i] || (km == key[i] && om < off[i]);
            rank[i] += lt ? 1 : 0;
        }
    }
}

// Final selection over the first nslots lane-strided slots, nb of which are
// members (non-members carry key +inf and rank after every member):
// FP64 refinement at the K-th boundary, then write ranks < K.
template <int N>
__device__ void select_and_write(const RerankParams& P, const float* ref, double (&key)[N],
                                 int (&off)[N], int nslots, int nb, int lane, size_t r,
                                 float gamma) {
    int rank[N];
    rank_members(key, off, nslots, lane, rank);
    if (nb > P.K) {
        // distances at ranks K-1 (last in) and K (first out), broadcast to the warp
        double din = 0.0, dout = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const bool m = lane + 32 * i < nslots;
            din += (m && rank[i] == P.K - 1) ? key[i] : 0.0;
            dout += (m && rank[i] == P.K) ? key[i] : 0.0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            din += __shfl_xor_sync(0xffffffffu, din, o);
            dout += __shfl_xor_sync(0xffffffffu, dout, o);
        }
        const double tol = (double)gamma * (din + dout);
        if (dout - din <= tol) {
            int nrec = 0;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int m = lane + 32 * i;
                if (m < nslots && rank[i] < nb && key[i] >= din - 2.0 * tol &&
                    key[i] <= dout + 2.0 * tol) {
                    key[i] = direct_f64(P, ref, off[i] / P.W, off[i] % P.W);
                    ++nrec;
                }
            }
            for (int o = 16; o > 0; o >>= 1) nrec += __shfl_xor_sync(0xffffffffu, nrec, o);
            if (lane == 0 && nrec) atomicAdd(P.counters + 1, (unsigned long long)nrec);
            rank_members(key, off, nslots, lane, rank);
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int m = lane + 32 * i;
        if (m < nslots && rank[i] < nb && rank[i] < P.K) {
            P.out_idx[r * P.K + rank[i]] = off[i];
            P.out_dist[r * P.K + rank[i]] = (float)key[i];
        }
    }
    for (int k = nb + lane; k < P.K; k += 32) {
        P.out_idx[r * P.K + k] = -1;
        P.out_dist[r * P.K + k] = __int_as_float(0x7f800000);
    }
}

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
    float v[kSlots];
    int off[kSlots];
    float nc[kSlots];
    int npool = 0;
#pragma unroll
    for (int i = 0; i < kSlots; ++i) {
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
    bool member[kSlots];
#pragma unroll
    for (int i = 0; i < kSlots; ++i) member[i] = off[i] >= 0;
    int nb = npool;
    bool overflow = false;
    if (npool > P.K) {
        // rank of every entry by v descending (ties: slot order)
        int rk[kSlots];
#pragma unroll
        for (int i = 0; i < kSlots; ++i) rk[i] = 0;
        for (int m = 0; m < P.L; ++m) {
            const int src = m & 31, slot = m >> 5;
            float vm = v[0];
#pragma unroll
            for (int k = 1; k < kSlots; ++k) vm = slot == k ? v[k] : vm;
            vm = __shfl_sync(0xffffffffu, vm, src);
#pragma unroll
            for (int i = 0; i < kSlots; ++i) {
                const int me = lane + 32 * i;
                rk[i] += (vm > v[i] || (vm == v[i] && m < me)) ? 1 : 0;
            }
        }
        float vK = -__int_as_float(0x7f800000), ncmax = 0.f;
#pragma unroll
        for (int i = 0; i < kSlots; ++i) {
            if (off[i] >= 0 && rk[i] == P.K - 1) vK = v[i];
            if (off[i] >= 0 && rk[i] < P.K) ncmax = fmaxf(ncmax, nc[i]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            vK = fmaxf(vK, __shfl_xor_sync(0xffffffffu, vK, o));
            ncmax = fmaxf(ncmax, __shfl_xor_sync(0xffffffffu, ncmax, o));
        }
        const float tb = vK - 2.0f * kEps * (nr + ncmax) * 1.0001f;
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < kSlots; ++i) {
            member[i] = off[i] >= 0 && v[i] >= tb;
            cnt += member[i] ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        nb = cnt;
        overflow = (npool == P.L) && (nb == P.L);
    }

    if (!overflow) {
        double key[kSlots];
        int viol = 0;
#pragma unroll
        for (int i = 0; i < kSlots; ++i) {
            key[i] = __longlong_as_double(0x7ff0000000000000ll);  // +inf: not a member
            if (member[i]) {
                const float d32 = direct_f32(P, ref, off[i] / P.W, off[i] % P.W);
                key[i] = d32;
                // identity estimate d~ = n_r - 2 (v - eps n_j) against its bound 2 eps (n_r + n_j)
                const float dt = nr - 2.0f * (v[i] - kEps * nc[i]);
                if (fabsf(dt - d32) > 2.0f * kEps * (nr + nc[i]) + gamma * d32 + 1e-6f * (nr + nc[i]) + 1.0f) ++viol;
            } else {
                off[i] = 0x7fffffff;
            }
        }
        for (int o = 16; o > 0; o >>= 1) viol += __shfl_xor_sync(0xffffffffu, viol, o);
        if (lane == 0 && viol) atomicAdd(P.counters + 2, (unsigned long long)viol);
        select_and_write(P, ref, key, off, P.L, nb, lane, r, gamma);
        return;
    }

    // ---- overflow: exact top-(K+1) over the whole window, FP32 direct distances
    if (lane == 0) atomicAdd(P.counters + 0, 1ull);
    unsigned long long* list = list_s[warp];
    const int nl = P.K + 1;
    for (int e = lane; e < kFbSlots * 32; e += 32) list[e] = ~0ull;
    __syncwarp();
    const int Hc = P.H - P.p + 1;
    const int y0 = max(0, yr - P.h), y1 = min(Hc - 1, yr + P.h);
    const int x0 = max(0, xr - P.h), x1 = min(P.Wc - 1, xr + P.h);
    const int nxw = x1 - x0 + 1;
    const int total = (y1 - y0 + 1) * nxw;
    for (int base = 0; base < total; base += 32) {
        const int i = base + lane;
        unsigned long long key = ~0ull;
        if (i < total) {
            const int yc = y0 + i / nxw, xc = x0 + i % nxw;
            const float d = direct_f32(P, ref, yc, xc);
            key = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(yc * P.W + xc);
        }
        unsigned pass = __ballot_sync(0xffffffffu, key < list[nl - 1]);
        while (pass) {
            const int src = __ffs(pass) - 1;
            pass &= pass - 1;
            const unsigned long long k = __shfl_sync(0xffffffffu, key, src);
            if (!(k < list[nl - 1])) continue;
            int pos = 0;
            for (int e = lane; e < nl; e += 32) pos += list[e] < k ? 1 : 0;
            for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
            unsigned long long nv[kFbSlots];
#pragma unroll
            for (int t = 0; t < kFbSlots; ++t) {
                const int e = lane + 32 * t;
                nv[t] = e < nl ? (e > pos ? list[e - 1] : (e == pos ? k : list[e])) : ~0ull;
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kFbSlots; ++t)
                if (lane + 32 * t < nl) list[lane + 32 * t] = nv[t];
            __syncwarp();
        }
    }
    double key2[kFbSlots];
    int off2[kFbSlots];
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < kFbSlots; ++t) {
        const int e = lane + 32 * t;
        const unsigned long long k = e < nl ? list[e] : ~0ull;
        key2[t] = k == ~0ull ? 0.0 : (double)__uint_as_float((unsigned)(k >> 32));
        off2[t] = k == ~0ull ? -1 : (int)(unsigned)(k & 0xffffffffu);
        cnt += (k != ~0ull) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    select_and_write(P, ref, key2, off2, cnt, cnt, lane, r, gamma);
}

}  // namespace

cudaError_t launch_rerank(const Geom& g, const float* img, const float* nrm,
                          const int32_t* pool_idx, const float* pool_score, int32_t* out_idx,
                          float* out_dist, unsigned long long* counters, cudaStream_t st) {
    if (g.L > kMaxPool) return cudaErrorNotSupported;
    RerankParams P{};
    P.img = img; P.nrm = nrm; P.pool_idx = pool_idx; P.pool_score = pool_score;
    P.out_idx = out_idx; P.out_dist = out_dist; P.counters = counters;
    P.H = g.H; P.W = g.W; P.C = g.C; P.p = g.p; P.h = g.h; P.s = g.s; P.K = g.K; P.L = g.L;
    P.n_ry = g.n_ry; P.n_rx = g.n_rx; P.Wc = g.Wc; P.nR = g.nR;
    const int blocks = (g.nR + kWarps - 1) / kWarps;
    rerank_kernel<<<blocks, kWarps * 32, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace bm
