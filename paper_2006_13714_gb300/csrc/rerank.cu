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
// memory, so every distance reads shared memory.  One warp per reference;
// every ranking uses 64-bit integer keys (FP64 is slow on this part and is
// kept to the rare boundary ties).  Shapes whose region does not fit run
// the same steps on global memory, one image per launch.
#include "bm_internal.h"

#include <climits>

namespace bm {
namespace {

constexpr float kEps = 6.103515625e-05f;  // 2^-14, same constant as the tensor-core pass
constexpr int kFbSlots = (kMaxK + 1 + 31) / 32;
constexpr unsigned long long kNone = ~0ull;
constexpr int kTileWarps = 8;
constexpr int kMaxRerankJobs = 64;
constexpr int kTileSmemLimit = 160 * 1024;

struct RerankJob {
    const float* img;
    const float* nrm;
    const int32_t* pool_idx;
    const float* pool_score;
    int32_t* out_idx;
    float* out_dist;
    int H, W, n_ry, n_rx, Hc, Wc;
    int tiles_x, tile_begin;
};

struct RerankParams {
    int C, p, h, s, K, L;
    float round_rel;  // pool-score rounding, relative: 2^(tbits - 23) (0: exact scores)
    float gamma;      // FP32 relative error bound of a direct distance
    int TRY, TRX;     // references per tile (rows, columns)
    int img_cap;      // shared-memory image region capacity (floats); norms follow
    unsigned long long* counters;  // [0] overflow, [1] fp64 rechecks, [2] bound violations
    int njobs, total_tiles;
    RerankJob jobs[kMaxRerankJobs];
};

// Pixel source: a region of the image (shared memory) or the whole image;
// element (y, x, c) at base + (y - y0) * pitch + (x - x0) * C + c.
struct Pix {
    const float* base;
    int y0, x0, pitch, C;
    __device__ __forceinline__ const float* at(int y, int x) const {
        return base + (size_t)(y - y0) * pitch + (size_t)(x - x0) * C;
    }
};

// (X_r - X_j)^2 summed row by row, elements in order (the reference's rows
// at ref + u * pitch).
__device__ __forceinline__ float direct_f32(const Pix& X, int p, int C, const float* ref, int yc, int xc) {
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

__device__ __forceinline__ double direct_f64(const Pix& X, int p, int C, const float* ref, int yc, int xc) {
    const int pc = p * C;
    double acc = 0.0;
    for (int u = 0; u < p; ++u) {
        const float* crow = X.at(yc + u, xc);
        const float* rrow = ref + (size_t)u * X.pitch;
        for (int e = 0; e < pc; ++e) {
            const double d = (double)rrow[e] - (double)crow[e];
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

// Final selection: members carry key (float(d32) bits << 32 | offset);
// non-members carry kNone.  FP64 refinement at the K-th boundary, then write
// ranks < K (and the padding).
template <int S>
__device__ void select_and_write(const RerankParams& P, const RerankJob& J, const Pix& X,
                                 const float* ref, const unsigned long long (&key)[S], int nb,
                                 int lane, size_t r) {
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
        const float tol = P.gamma * (din + dout);
        if (dout - din <= tol) {
            // boundary members: FP64 distances decide their order
            int nrec = 0;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const float d = __uint_as_float((unsigned)(key[i] >> 32));
                if (key[i] != kNone && d >= din - 2.f * tol && d <= dout + 2.f * tol) {
                    const int off = (int)(unsigned)(key[i] & 0xffffffffu);
                    d64[i] = direct_f64(X, P.p, P.C, ref, off / J.W, off % J.W);
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

// The steps of the file header for reference (ry, rx) of job J.  X holds
// every pixel of the patches of its window, N (C = 1) every norm of its
// window; list: kFbSlots * 32 words of shared memory for the overflow path.
template <int S>
__device__ void rerank_ref(const RerankParams& P, const RerankJob& J, const Pix& X, const Pix& N,
                           int ry, int rx, int lane, unsigned long long* list) {
    const size_t r = (size_t)ry * J.n_rx + rx;
    const int yr = ry * P.s, xr = rx * P.s;
    const float* ref = X.at(yr, xr);  // reference rows at ref + u * X.pitch
    const float nr = *N.at(yr, xr);

    // ---- load the pool (best first; empty slots have offset -1)
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
            off[i] = J.pool_idx[r * P.L + k];
            if (off[i] >= 0) {
                v[i] = J.pool_score[r * P.L + k];
                nc[i] = *N.at(off[i] / J.W, off[i] % J.W);
                ++npool;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) npool += __shfl_xor_sync(0xffffffffu, npool, o);

    // ---- band: entries with v >= tb (see the file header); the pool is
    // sorted, so the K-th largest score is entry K-1
    bool member[S];
#pragma unroll
    for (int i = 0; i < S; ++i) member[i] = off[i] >= 0;
    int nb = npool;
    bool overflow = false;
    if (npool > P.K) {
        float vK = -__int_as_float(0x7f800000), ncmax = 0.f, vabs = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const int k = lane + 32 * i;
            if (k == P.K - 1) vK = v[i];
            if (k < P.K) {
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
                const float d32 = direct_f32(X, P.p, P.C, ref, off[i] / J.W, off[i] % J.W);
                key[i] = ((unsigned long long)__float_as_uint(d32) << 32) | (unsigned)off[i];
                // identity estimate d~ = n_r - 2 (v - eps n_j) against its bound 2 eps (n_r + n_j)
                const float dt = nr - 2.0f * (v[i] - kEps * nc[i]);
                if (fabsf(dt - d32) > 2.0f * kEps * (nr + nc[i]) + 2.0f * P.round_rel * fabsf(v[i]) +
                                          P.gamma * d32 + 1e-6f * (nr + nc[i]) + 1.0f)
                    ++viol;
            }
        }
        for (int o = 16; o > 0; o >>= 1) viol += __shfl_xor_sync(0xffffffffu, viol, o);
        if (lane == 0 && viol) atomicAdd(P.counters + 2, (unsigned long long)viol);
        select_and_write<S>(P, J, X, ref, key, nb, lane, r);
        return;
    }

    // ---- overflow: exact top-(K+1) over the whole window, FP32 direct distances
    if (lane == 0) atomicAdd(P.counters + 0, 1ull);
    const int nl = P.K + 1;
    for (int e = lane; e < kFbSlots * 32; e += 32) list[e] = kNone;
    __syncwarp();
    const int y0 = max(0, yr - P.h), y1 = min(J.Hc - 1, yr + P.h);
    const int x0 = max(0, xr - P.h), x1 = min(J.Wc - 1, xr + P.h);
    const int nxw = x1 - x0 + 1;
    const int total = (y1 - y0 + 1) * nxw;
    for (int base = 0; base < total; base += 32) {
        const int i = base + lane;
        unsigned long long k = kNone;
        if (i < total) {
            const int yc = y0 + i / nxw, xc = x0 + i % nxw;
            const float d = direct_f32(X, P.p, P.C, ref, yc, xc);
            k = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(yc * J.W + xc);
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
    select_and_write<kFbSlots>(P, J, X, ref, key2, cnt, lane, r);
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

template <int S>
__global__ void __launch_bounds__(kTileWarps * 32) rerank_tile_kernel(const __grid_constant__ RerankParams P) {
    extern __shared__ __align__(16) float sm[];
    __shared__ unsigned long long list_s[kTileWarps][kFbSlots * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x;
    const RerankJob& J = P.jobs[tile_job(P, t)];
    const int lt = t - J.tile_begin;
    const int ry0 = (lt / J.tiles_x) * P.TRY, rx0 = (lt % J.tiles_x) * P.TRX;
    const int ry1 = min(ry0 + P.TRY, J.n_ry) - 1, rx1 = min(rx0 + P.TRX, J.n_rx) - 1;
    // region: every pixel of every window patch of the tile's references
    const int iy0 = max(0, ry0 * P.s - P.h), iy1 = min(J.H - 1, ry1 * P.s + P.h + P.p - 1);
    const int ix0 = max(0, rx0 * P.s - P.h), ix1 = min(J.W - 1, rx1 * P.s + P.h + P.p - 1);
    const int ny1 = min(J.Hc - 1, ry1 * P.s + P.h), nx1 = min(J.Wc - 1, rx1 * P.s + P.h);
    const int ipitch = (ix1 - ix0 + 1) * P.C, npitch = nx1 - ix0 + 1;
    float* simg = sm;
    float* snrm = sm + P.img_cap;
    const int irows = iy1 - iy0 + 1, nrows = ny1 - iy0 + 1;
    for (int i = threadIdx.x; i < irows * ipitch; i += blockDim.x) {
        const int y = i / ipitch, e = i % ipitch;
        simg[i] = __ldg(J.img + ((size_t)(iy0 + y) * J.W + ix0) * P.C + e);
    }
    for (int i = threadIdx.x; i < nrows * npitch; i += blockDim.x) {
        const int y = i / npitch, x = i % npitch;
        snrm[i] = __ldg(J.nrm + (size_t)(iy0 + y) * J.Wc + ix0 + x);
    }
    __syncthreads();
    const Pix X{simg, iy0, ix0, ipitch, P.C};
    const Pix N{snrm, iy0, ix0, npitch, 1};
    const int ncols = rx1 - rx0 + 1;
    const int nref = (ry1 - ry0 + 1) * ncols;
    for (int i = warp; i < nref; i += kTileWarps)
        rerank_ref<S>(P, J, X, N, ry0 + i / ncols, rx0 + i % ncols, lane, list_s[warp]);
}

// The same steps on global memory: one image, one reference per warp.
template <int S>
__global__ void __launch_bounds__(128) rerank_global_kernel(const __grid_constant__ RerankParams P) {
    __shared__ unsigned long long list_s[4][kFbSlots * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RerankJob& J = P.jobs[0];
    const size_t r = (size_t)blockIdx.x * 4 + warp;
    if (r >= (size_t)J.n_ry * J.n_rx) return;
    const Pix X{J.img, 0, 0, J.W * P.C, P.C};
    const Pix N{J.nrm, 0, 0, J.Wc, 1};
    rerank_ref<S>(P, J, X, N, (int)(r / J.n_rx), (int)(r % J.n_rx), lane, list_s[warp]);
}

// Tile shape and shared memory for a class; false: no region fits.
bool tile_shape(const Geom& g, int& TRY, int& TRX, int& img_cap, int& smem) {
    static const int kShapes[5][2] = {{8, 8}, {4, 8}, {4, 4}, {2, 2}, {1, 1}};
    for (const auto& sh : kShapes) {
        const int rows = (sh[0] - 1) * g.s + 2 * g.h + g.p;
        const int cols = (sh[1] - 1) * g.s + 2 * g.h + g.p;
        img_cap = (rows * cols * g.C + 3) / 4 * 4;
        smem = (img_cap + rows * cols) * 4;
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
    if (tiled) {
        cudaFuncSetAttribute(rerank_tile_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        rerank_tile_kernel<S><<<grid, kTileWarps * 32, smem, st>>>(P);
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
