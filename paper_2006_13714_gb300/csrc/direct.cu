// direct.cu -- plain FP32 CUDA-core direct-distance block matcher.
//
// The comparison baseline: every distance is the explicit sum of squared
// differences of Eq. equ:bmMetric_app (§III-E), summed over channels (§IV),
// in FP32 on the CUDA cores -- no Self-Convolution identity, no tensor
// cores.  One thread per reference patch; a warp holds one row of 32
// references, a block TRy warps, and the union of their search windows is
// staged in shared memory (or, when that union is too large, read through
// L1).  For patch sides 7 and 8, 1 or 4 channels and windows 21, 39 and 61
// the window row is register-blocked (all 2h+1 candidates of one candidate
// row accumulate together, so one load feeds 2h+1 fused multiply-adds);
// other shapes use a generic loop.  For uint8 the FP32 sums are exact (all
// partial sums are integers below 2^24), so results are bit-exact.
//
// Selection keeps the K smallest keys (distance, row-major offset) in a
// per-thread max-heap in shared memory; the output is sorted ascending.
#include "bm_internal.h"

#include <cfloat>
#include <climits>

namespace bm {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ unsigned long long make_key(float d, int off) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)off;
}

// Max-heap of keys, element i of thread t at heap[i * nthr + t].
struct ThreadHeap {
    unsigned long long* h;
    int nthr, K;
    __device__ void init(unsigned long long* base, int t, int nthreads, int k) {
        h = base + t;
        nthr = nthreads;
        K = k;
        for (int i = 0; i < K; ++i) h[i * nthr] = kEmptyKey;
    }
    __device__ void replace_top(unsigned long long key) {
        int i = 0;
        while (true) {
            int l = 2 * i + 1;
            if (l >= K) break;
            int r = l + 1;
            unsigned long long lv = h[l * nthr];
            int c = l;
            unsigned long long cv = lv;
            if (r < K) {
                unsigned long long rv = h[r * nthr];
                if (rv > lv) { c = r; cv = rv; }
            }
            if (cv <= key) break;
            h[i * nthr] = cv;
            i = c;
        }
        h[i * nthr] = key;
    }
    __device__ __forceinline__ void push(unsigned long long key) {
        if (key < h[0]) replace_top(key);
    }
    // In-place heap sort to ascending order, then write the output row.
    __device__ void emit(bool u8, int32_t* idx, void* dist) {
        for (int n = K - 1; n > 0; --n) {
            unsigned long long mx = h[0];
            unsigned long long last = h[n * nthr];
            h[n * nthr] = mx;
            int saveK = K;
            K = n;
            replace_top(last);
            K = saveK;
        }
        for (int k = 0; k < K; ++k) {
            unsigned long long key = h[k * nthr];
            if (key == kEmptyKey) {
                idx[k] = -1;
                if (u8) static_cast<int32_t*>(dist)[k] = INT_MAX;
                else static_cast<float*>(dist)[k] = __int_as_float(0x7f800000);
            } else {
                idx[k] = (int32_t)(unsigned)(key & 0xffffffffu);
                float d = __uint_as_float((unsigned)(key >> 32));
                if (u8) static_cast<int32_t*>(dist)[k] = (int32_t)d;
                else static_cast<float*>(dist)[k] = d;
            }
        }
    }
};

// Per-thread append buffer in front of the heap: keys below the current
// threshold are appended with predicated stores; when any lane of the warp
// nears a full buffer, the whole warp merges in lock-step (no divergent
// heap work per candidate).  Loops around it are warp-uniform.
constexpr int kBufD = 64;

struct BufferedTopK {
    ThreadHeap heap;
    unsigned long long* buf;  // element i at buf[i * nthr]
    int nthr, cnt;
    unsigned long long thr;
    __device__ void init(unsigned long long* heap_base, unsigned long long* buf_base, int t,
                         int nthreads, int K) {
        heap.init(heap_base, t, nthreads, K);
        buf = buf_base + t;
        nthr = nthreads;
        cnt = 0;
        thr = kEmptyKey;
    }
    __device__ __forceinline__ void append(unsigned long long key, bool valid) {
        if (valid && key < thr) {
            buf[cnt * nthr] = key;
            ++cnt;
        }
    }
    // warp-uniform call
    __device__ void merge() {
        const int m = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
        for (int j = 0; j < m; ++j)
            if (j < cnt) heap.push(buf[j * nthr]);
        cnt = 0;
        thr = heap.h[0];
    }
    __device__ __forceinline__ void make_room(int need) {
        if (__any_sync(0xffffffffu, cnt > kBufD - need)) merge();
    }
};

struct DirectParams {
    const void* img;
    int H, W, C, p, h, s, K, n_ry, n_rx, TRy;
    int Y_lo, X_lo;  // unused placeholders (per block)
    int32_t* out_idx;
    void* out_dist;
};

// Stage image rows [Yl, Yl+TY) x pixels [Xl, Xl+TX) (x C) as FP32, zero outside.
template <bool kU8>
__device__ void stage_tile(const DirectParams& P, float* tile, int Yl, int Xl, int TY, int TX) {
    const int row_f = TX * P.C;
    const int total = TY * row_f;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        int ty = i / row_f, e = i % row_f;
        int y = Yl + ty, x = Xl + e / P.C, c = e % P.C;
        float v = 0.f;
        if (y >= 0 && y < P.H && x >= 0 && x < P.W) {
            size_t src = ((size_t)y * P.W + x) * P.C + c;
            v = kU8 ? (float)static_cast<const uint8_t*>(P.img)[src]
                    : static_cast<const float*>(P.img)[src];
        }
        tile[i] = v;
    }
}

// Register-blocked kernel for a compile-time patch P, channels C, window NX.
// kG: read the image from global memory (through L1) instead of a staged
// tile -- for unions too large to stage; the shared memory then holds only
// the selection state, so more warps fit on an SM.
template <int PP, int CC, int NX, bool kU8, bool kG>
__global__ void __launch_bounds__(128)
direct_tpl_kernel(DirectParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int h = NX / 2;
    const int TRy = P.TRy;
    const int ry0 = blockIdx.y * TRy, rx0 = blockIdx.x * 32;
    const int Yl = ry0 * P.s - h, Xl = rx0 * P.s - h;
    const int TY = (TRy - 1) * P.s + NX + PP - 1;
    const int TX = 31 * P.s + NX + PP - 1;
    float* tile = reinterpret_cast<float*>(smem);
    size_t tile_bytes = kG ? 0 : ((size_t)TY * TX * CC * 4 + 15) & ~size_t(15);
    unsigned long long* heaps = reinterpret_cast<unsigned long long*>(smem + tile_bytes);
    unsigned long long* bufs = heaps + (size_t)blockDim.x * P.K;
    if (!kG) stage_tile<kU8>(P, tile, Yl, Xl, TY, TX);
    BufferedTopK top;
    top.init(heaps, bufs, threadIdx.x, blockDim.x, P.K);
    __syncthreads();

    const int ry = ry0 + threadIdx.x / 32, rx = rx0 + threadIdx.x % 32;
    if (ry >= P.n_ry) return;  // whole warp (one reference row per warp)
    const bool lane_ok = rx < P.n_rx;
    const int yr = ry * P.s, xr = min(rx, P.n_rx - 1) * P.s;
    const int Hc = P.H - PP + 1, Wc = P.W - PP + 1;
    const int rowf = TX * CC;
    // image element (y, x, c) as float, zero outside the image (global source)
    auto px = [&](int y, int x, int c) -> float {
        if (x < 0 || x >= P.W) return 0.f;
        const size_t i = ((size_t)y * P.W + x) * CC + c;
        return kU8 ? (float)__ldg(static_cast<const uint8_t*>(P.img) + i)
                   : __ldg(static_cast<const float*>(P.img) + i);
    };
    const int ylo = max(0, yr - h), yhi = min(Hc - 1, yr + h);  // warp-uniform
    for (int y = ylo; y <= yhi; ++y) {
        float acc[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) acc[i] = 0.f;
#pragma unroll 1
        for (int u = 0; u < PP; ++u) {
            const float* trow = tile + (size_t)(y - Yl + u) * rowf + (xr - h - Xl) * CC;
            const float* rrow = tile + (size_t)(yr - Yl + u) * rowf + (xr - Xl) * CC;
            // channels unrolled up to window 39; wider windows take them one at
            // a time (one candidate row of registers, no spills)
            constexpr int kCU = NX <= 39 ? CC : 1;
#pragma unroll kCU
            for (int c = 0; c < CC; ++c) {
                float t[NX + PP - 1];
#pragma unroll
                for (int i = 0; i < NX + PP - 1; ++i)
                    t[i] = kG ? px(y + u, xr - h + i, c) : trow[i * CC + c];
#pragma unroll
                for (int v = 0; v < PP; ++v) {
                    const float r = kG ? px(yr + u, xr + v, c) : rrow[v * CC + c];
#pragma unroll
                    for (int i = 0; i < NX; ++i) {
                        float d = r - t[i + v];
                        acc[i] = fmaf(d, d, acc[i]);
                    }
                }
            }
        }
        top.make_room(NX);
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            const int x = xr - h + i;
            top.append(make_key(acc[i], y * P.W + x), lane_ok && x >= 0 && x < Wc);
        }
    }
    top.merge();
    if (!lane_ok) return;
    size_t ref = (size_t)ry * P.n_rx + rx;
    top.heap.emit(kU8, P.out_idx + ref * P.K,
                  kU8 ? (void*)(static_cast<int32_t*>(P.out_dist) + ref * P.K)
                      : (void*)(static_cast<float*>(P.out_dist) + ref * P.K));
}

// Generic kernel: runtime patch / channels / window, one candidate at a time.
// kTile selects the shared-memory union tile; otherwise pixels come from global.
template <bool kU8, bool kTile>
__global__ void __launch_bounds__(128)
direct_generic_kernel(DirectParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int h = P.h, pp = P.p, C = P.C;
    const int TRy = P.TRy;
    const int ry0 = blockIdx.y * TRy, rx0 = blockIdx.x * 32;
    const int NX = 2 * h + 1;
    const int Yl = ry0 * P.s - h, Xl = rx0 * P.s - h;
    const int TY = (TRy - 1) * P.s + NX + pp - 1;
    const int TX = 31 * P.s + NX + pp - 1;
    float* tile = reinterpret_cast<float*>(smem);
    size_t tile_bytes = kTile ? (((size_t)TY * TX * C * 4 + 15) & ~size_t(15)) : 0;
    unsigned long long* heaps = reinterpret_cast<unsigned long long*>(smem + tile_bytes);
    unsigned long long* bufs = heaps + (size_t)blockDim.x * P.K;
    if (kTile) stage_tile<kU8>(P, tile, Yl, Xl, TY, TX);
    BufferedTopK top;
    top.init(heaps, bufs, threadIdx.x, blockDim.x, P.K);
    __syncthreads();
    const int ry = ry0 + threadIdx.x / 32, rx = rx0 + threadIdx.x % 32;
    if (ry >= P.n_ry) return;  // whole warp
    const bool lane_ok = rx < P.n_rx;
    const int yr = ry * P.s, xr = rx * P.s;
    const int Hc = P.H - pp + 1, Wc = P.W - pp + 1;
    const int ylo = max(0, yr - h), yhi = min(Hc - 1, yr + h);  // warp-uniform
    const int rowf = TX * C;
    for (int y = ylo; y <= yhi; ++y) {
        for (int dx = -h; dx <= h; ++dx) {  // warp-uniform
            const int x = xr + dx;
            const bool ok = lane_ok && x >= 0 && x < Wc;
            float acc = 0.f;
            if (ok) {
                for (int u = 0; u < pp; ++u) {
                    for (int e = 0; e < pp * C; ++e) {
                        float a, b;
                        if (kTile) {
                            a = tile[(size_t)(yr - Yl + u) * rowf + (xr - Xl) * C + e];
                            b = tile[(size_t)(y - Yl + u) * rowf + (x - Xl) * C + e];
                        } else {
                            size_t ia = ((size_t)(yr + u) * P.W + xr) * C + e;
                            size_t ib = ((size_t)(y + u) * P.W + x) * C + e;
                            a = kU8 ? (float)__ldg(static_cast<const uint8_t*>(P.img) + ia)
                                    : __ldg(static_cast<const float*>(P.img) + ia);
                            b = kU8 ? (float)__ldg(static_cast<const uint8_t*>(P.img) + ib)
                                    : __ldg(static_cast<const float*>(P.img) + ib);
                        }
                        float d = a - b;
                        acc = fmaf(d, d, acc);
                    }
                }
            }
            top.make_room(1);
            top.append(make_key(acc, y * P.W + x), ok);
        }
    }
    top.merge();
    if (!lane_ok) return;
    size_t ref = (size_t)ry * P.n_rx + rx;
    top.heap.emit(kU8, P.out_idx + ref * P.K,
                  kU8 ? (void*)(static_cast<int32_t*>(P.out_dist) + ref * P.K)
                      : (void*)(static_cast<float*>(P.out_dist) + ref * P.K));
}

size_t direct_smem(const Geom& g, int TRy, bool tile) {
    int NX = 2 * g.h + 1;
    int TY = (TRy - 1) * g.s + NX + g.p - 1;
    int TX = 31 * g.s + NX + g.p - 1;
    size_t tb = tile ? (((size_t)TY * TX * g.C * 4 + 15) & ~size_t(15)) : 0;
    return tb + (size_t)TRy * 32 * (g.K + kBufD) * 8;
}

template <int PP, int CC, int NX, bool kG>
cudaError_t launch_tpl(const DirectParams& P, dim3 grid, size_t sm, bool u8, cudaStream_t st) {
    if (u8) {
        auto k = direct_tpl_kernel<PP, CC, NX, true, kG>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<grid, P.TRy * 32, sm, st>>>(P);
    } else {
        auto k = direct_tpl_kernel<PP, CC, NX, false, kG>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<grid, P.TRy * 32, sm, st>>>(P);
    }
    return cudaGetLastError();
}

// Register-blocked instance for (p, C, window), if one exists.
template <bool kG>
bool launch_tpl_any(const Geom& g, const DirectParams& P, dim3 grid, size_t sm, bool u8,
                    cudaStream_t st, cudaError_t* e) {
    const int NX = 2 * g.h + 1;
#define BM_DIRECT_CASE(PP, CC, WW)                                          \
    if (g.p == PP && g.C == CC && NX == WW) {                                \
        *e = launch_tpl<PP, CC, WW, kG>(P, grid, sm, u8, st);                \
        return true;                                                         \
    }
    BM_DIRECT_CASE(8, 1, 21)
    BM_DIRECT_CASE(8, 1, 39)
    BM_DIRECT_CASE(8, 1, 61)
    BM_DIRECT_CASE(7, 1, 39)
    BM_DIRECT_CASE(7, 1, 61)
    BM_DIRECT_CASE(8, 4, 39)
    BM_DIRECT_CASE(8, 4, 61)
    BM_DIRECT_CASE(7, 4, 39)
    BM_DIRECT_CASE(7, 4, 61)
#undef BM_DIRECT_CASE
    return false;
}

}  // namespace

cudaError_t launch_direct(const Geom& g, const void* img, int32_t* out_idx, void* out_dist,
                          cudaStream_t st) {
    DirectParams P{};
    P.img = img;
    P.H = g.H; P.W = g.W; P.C = g.C; P.p = g.p; P.h = g.h; P.s = g.s; P.K = g.K;
    P.n_ry = g.n_ry; P.n_rx = g.n_rx;
    P.out_idx = out_idx;
    P.out_dist = out_dist;
    const size_t kSmemCap = 200 * 1024;
    const bool u8 = g.dtype == kU8;
    {
        // register-blocked: a staged union tile when two or more warps of
        // references fit, else the image through L1 with four warps
        int TRy = 4;
        while (TRy > 2 && direct_smem(g, TRy, true) > kSmemCap) TRy /= 2;
        const bool staged = direct_smem(g, TRy, true) <= kSmemCap;
        if (!staged) TRy = 4;
        P.TRy = TRy;
        const size_t sm = direct_smem(g, TRy, staged);
        dim3 grid((g.n_rx + 31) / 32, (g.n_ry + TRy - 1) / TRy);
        cudaError_t e = cudaSuccess;
        if (staged ? launch_tpl_any<false>(g, P, grid, sm, u8, st, &e)
                   : launch_tpl_any<true>(g, P, grid, sm, u8, st, &e))
            return e;
    }
    int TRy = 4;
    bool tile = true;
    while (TRy > 1 && direct_smem(g, TRy, true) > kSmemCap) TRy /= 2;
    if (direct_smem(g, TRy, true) > kSmemCap) {
        tile = false;
        TRy = 4;
        while (TRy > 1 && direct_smem(g, TRy, false) > kSmemCap) TRy /= 2;
    }
    P.TRy = TRy;
    size_t sm = direct_smem(g, TRy, tile);
    dim3 grid((g.n_rx + 31) / 32, (g.n_ry + TRy - 1) / TRy);
    if (u8) {
        auto k = tile ? direct_generic_kernel<true, true> : direct_generic_kernel<true, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<grid, TRy * 32, sm, st>>>(P);
    } else {
        auto k = tile ? direct_generic_kernel<false, true> : direct_generic_kernel<false, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<grid, TRy * 32, sm, st>>>(P);
    }
    return cudaGetLastError();
}

}  // namespace bm
