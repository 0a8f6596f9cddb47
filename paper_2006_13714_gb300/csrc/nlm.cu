// nlm.cu -- non-local means weights and patch estimates (§III-A, Eq. equ:nlm;
// Prop. 1 gives the same weights through Self-Convolution), windowed like
// block matching (footnote to Eq. eq:unifySelfConv).
//
// For every reference patch X_r of the stride grid and every candidate X_j
// of its clipped search window:
//   w_r(j) = exp(-||X_j - X_r||^2 / b^2),   Theta_r = sum_j w_r(j),
//   Xhat_r = sum_j w_r(j) X_j / Theta_r      (the NLM estimate of X_r).
// The reference is its own candidate (distance 0, weight 1), so every
// weight is at most 1 and Theta_r >= 1: no running maximum is needed.
//
// GB300 layout of the work (CUDA cores, FP32).  One block per tile of up to
// 8 x 8 references; the image region their windows cover is staged in shared
// memory as element pairs (pair e of a row holds elements e and e + 1), so a
// patch row starting anywhere is read with 64-bit loads and processed two
// elements at a time with packed FP32 arithmetic (sub/fma.rn.f32x2).  The
// region's row pitch is the window width times C mod 16 pairs: 32 candidates
// that wrap onto the next window row still read distinct banks.  One
// warp per reference, one lane per candidate (strided over the window): the
// lane forms the distance, its weight (ex2), and adds the weighted candidate
// into its register copy of the estimate; a butterfly over the warp sums the
// 32 partial estimates.  Work per reference and candidate: 2 p^2 C FLOP for
// the distance plus 2 p^2 C for the weighted sum (ALU-bound).
#include "bm.h"
#include "bm_internal.h"

#include <algorithm>
#include <string>

namespace bm {
namespace {

constexpr int kNlmThreads = 256;
constexpr int kNlmMaxPatchElems = 64;        // p*p*C served (register estimate)
constexpr int kNlmSmemLimit = 160 * 1024;

struct NlmParams {
    const void* img;
    float* est;           // [n_ry*n_rx][p*p*C]
    float* theta;         // nullable [n_ry*n_rx]
    int H, W, C, p, h, s, n_ry, n_rx, Hc, Wc;
    int dtype;
    int ty, tx, tiles_x;  // references per tile (rows, columns), tiles along x
    int rows, cols;       // staged region extent (pixels) for a full tile
    float k2;             // log2(e) / b^2
};

__device__ __forceinline__ unsigned long long pk(float2 v) {
    return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}
// An element pair straight from shared memory into a 64-bit register (the
// operand form of the packed FP32 instructions).
__device__ __forceinline__ unsigned long long ld2(const float2* q) {
    return *reinterpret_cast<const unsigned long long*>(q);
}
__device__ __forceinline__ float2 upk(unsigned long long v) {
    return make_float2(__uint_as_float((unsigned)v), __uint_as_float((unsigned)(v >> 32)));
}

// P, C: patch side and channels (compile time: the estimate lives in registers).
template <int P, int C>
__global__ void __launch_bounds__(kNlmThreads) nlm_kernel(const NlmParams Q) {
    constexpr int PC = P * C, NPR = PC / 2, TAIL = PC & 1;
    extern __shared__ __align__(16) float2 sreg[];
    const int ty = blockIdx.x / Q.tiles_x, tx = blockIdx.x - ty * Q.tiles_x;
    const int ry0 = ty * Q.ty, rx0 = tx * Q.tx;
    const int ry1 = min(ry0 + Q.ty, Q.n_ry) - 1, rx1 = min(rx0 + Q.tx, Q.n_rx) - 1;
    // region: every candidate patch of the tile's windows
    const int Y0 = max(0, ry0 * Q.s - Q.h), X0 = max(0, rx0 * Q.s - Q.h);
    const int Y1 = min(Q.Hc - 1, ry1 * Q.s + Q.h) + P, X1 = min(Q.Wc - 1, rx1 * Q.s + Q.h) + P;
    const int nrow = Y1 - Y0, width = (X1 - X0) * C;  // pairs per region row
    const int pitch = width + (((2 * Q.h + 1) * C - width) & 15);  // padded row pitch
    for (int i = threadIdx.x; i < nrow * width; i += blockDim.x) {
        const int r = i / width, e = i - r * width;
        const size_t g = ((size_t)(Y0 + r) * Q.W + X0) * C + e;
        float a, b;
        if (Q.dtype == kU8) {
            const uint8_t* im = static_cast<const uint8_t*>(Q.img);
            a = im[g];
            b = e + 1 < width ? im[g + 1] : 0.f;
        } else {
            const float* im = static_cast<const float*>(Q.img);
            a = im[g];
            b = e + 1 < width ? im[g + 1] : 0.f;
        }
        sreg[r * pitch + e] = make_float2(a, b);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int nref = (ry1 - ry0 + 1) * (rx1 - rx0 + 1);
    for (int rl = warp; rl < nref; rl += nwarps) {
        const int ry = ry0 + rl / (rx1 - rx0 + 1), rx = rx0 + rl % (rx1 - rx0 + 1);
        const int yr = ry * Q.s, xr = rx * Q.s;
        const int cy0 = max(0, yr - Q.h), cy1 = min(Q.Hc - 1, yr + Q.h);
        const int cx0 = max(0, xr - Q.h), cx1 = min(Q.Wc - 1, xr + Q.h);
        const int wx = cx1 - cx0 + 1, ncand = (cy1 - cy0 + 1) * wx;
        const float2* rb = sreg + (yr - Y0) * pitch + (xr - X0) * C;
        unsigned long long acc[P][NPR > 0 ? NPR : 1];
        float acct[P];
#pragma unroll
        for (int u = 0; u < P; ++u) {
#pragma unroll
            for (int t = 0; t < NPR; ++t) acc[u][t] = 0ull;
            acct[u] = 0.f;
        }
        float theta = 0.f;
        for (int j = lane; j < ncand; j += 32) {
            const int jy = j / wx, jx = j - jy * wx;
            const float2* cb = sreg + (cy0 + jy - Y0) * pitch + (cx0 + jx - X0) * C;
            // distance, two elements at a time, in two chains (even / odd patch rows)
            unsigned long long dd[2] = {0ull, 0ull};
            float dt = 0.f;
#pragma unroll
            for (int u = 0; u < P; ++u) {
#pragma unroll
                for (int t = 0; t < NPR; ++t) {
                    unsigned long long df;
                    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(ld2(&rb[u * pitch + 2 * t])), "l"(ld2(&cb[u * pitch + 2 * t])));
                    asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(dd[u & 1]) : "l"(df));
                }
                if (TAIL) {
                    const float df = rb[u * pitch + PC - 1].x - cb[u * pitch + PC - 1].x;
                    dt = fmaf(df, df, dt);
                }
            }
            const float2 d2 = upk(dd[0]), d3 = upk(dd[1]);
            const float d = ((d2.x + d2.y) + (d3.x + d3.y)) + dt;
            const float w = exp2f(-d * Q.k2);
            theta += w;
            unsigned long long ww;
            asm("mov.b64 %0, {%1, %1};" : "=l"(ww) : "f"(w));
#pragma unroll
            for (int u = 0; u < P; ++u) {
#pragma unroll
                for (int t = 0; t < NPR; ++t)
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[u][t]) : "l"(ww), "l"(ld2(&cb[u * pitch + 2 * t])));
                if (TAIL) acct[u] = fmaf(w, cb[u * pitch + PC - 1].x, acct[u]);
            }
        }
        // butterfly sum over the warp (every lane ends with the totals)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            theta += __shfl_xor_sync(0xffffffffu, theta, o);
#pragma unroll
            for (int u = 0; u < P; ++u) {
#pragma unroll
                for (int t = 0; t < NPR; ++t) {
                    const float2 a = upk(acc[u][t]);
                    acc[u][t] = pk(make_float2(a.x + __shfl_xor_sync(0xffffffffu, a.x, o),
                                               a.y + __shfl_xor_sync(0xffffffffu, a.y, o)));
                }
                if (TAIL) acct[u] += __shfl_xor_sync(0xffffffffu, acct[u], o);
            }
        }
        const size_t ref = (size_t)ry * Q.n_rx + rx;
        // lane u writes patch row u (rows beyond 32 by lane u - 32, ...)
        float* out = Q.est + ref * (P * PC);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            if ((u & 31) != lane) continue;
#pragma unroll
            for (int t = 0; t < NPR; ++t) {
                const float2 a = upk(acc[u][t]);
                out[u * PC + 2 * t] = a.x / theta;
                out[u * PC + 2 * t + 1] = a.y / theta;
            }
            if (TAIL) out[u * PC + PC - 1] = acct[u] / theta;
        }
        if (Q.theta && lane == 0) Q.theta[ref] = theta;
    }
}

using NlmKernel = void (*)(NlmParams);

// Instantiated (patch, channels) shapes; p*p*C <= 64.
NlmKernel pick_kernel(int p, int C) {
#define BM_NLM_CASE(PP, CC) \
    if (p == PP && C == CC) return nlm_kernel<PP, CC>;
    BM_NLM_CASE(1, 1) BM_NLM_CASE(2, 1) BM_NLM_CASE(3, 1) BM_NLM_CASE(4, 1) BM_NLM_CASE(5, 1)
    BM_NLM_CASE(6, 1) BM_NLM_CASE(7, 1) BM_NLM_CASE(8, 1)
    BM_NLM_CASE(1, 2) BM_NLM_CASE(2, 2) BM_NLM_CASE(3, 2) BM_NLM_CASE(4, 2) BM_NLM_CASE(5, 2)
    BM_NLM_CASE(1, 3) BM_NLM_CASE(2, 3) BM_NLM_CASE(3, 3) BM_NLM_CASE(4, 3)
    BM_NLM_CASE(1, 4) BM_NLM_CASE(2, 4) BM_NLM_CASE(3, 4) BM_NLM_CASE(4, 4)
    BM_NLM_CASE(1, 8) BM_NLM_CASE(2, 8)
#undef BM_NLM_CASE
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

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

int bm_nlm(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
           int window, int stride, float b, float* out_est, float* out_theta, bm_stream stream) {
    if (!ctx) return set_error(BM_ERR_INVALID, "null context");
    if (dtype != BM_U8 && dtype != BM_F32) return set_error(BM_ERR_INVALID, "unknown dtype");
    if (H < 1 || W < 1 || C < 1 || C > kMaxC || patch < 1 || patch > H || patch > W ||
        window < 1 || window % 2 == 0 || window > kMaxWindow || stride < 1)
        return set_error(BM_ERR_INVALID, "invalid geometry");
    if (!(b > 0.f) || !(b < 3.0e38f)) return set_error(BM_ERR_INVALID, "b must be positive and finite");
    if (!img || !out_est) return set_error(BM_ERR_INVALID, "null pointer");
    if ((long long)H * W >= (1LL << 31)) return set_error(BM_ERR_UNSUPPORTED, "H*W must be below 2^31");
    if (patch * patch * C > kNlmMaxPatchElems)
        return set_error(BM_ERR_UNSUPPORTED, "patch*patch*C must be at most 64 for NLM");
    const NlmKernel kern = pick_kernel(patch, C);
    if (!kern) return set_error(BM_ERR_UNSUPPORTED, "patch / channel shape not instantiated");
    NlmParams Q{};
    Q.img = img; Q.est = out_est; Q.theta = out_theta;
    Q.H = H; Q.W = W; Q.C = C; Q.p = patch; Q.h = (window - 1) / 2; Q.s = stride;
    Q.n_ry = (H - patch) / stride + 1; Q.n_rx = (W - patch) / stride + 1;
    Q.Hc = H - patch + 1; Q.Wc = W - patch + 1;
    Q.dtype = dtype == BM_U8 ? kU8 : kF32;
    Q.k2 = 1.4426950408889634f / (b * b);
    if (!(Q.k2 > 0.f)) return set_error(BM_ERR_UNSUPPORTED, "b too large (1/b^2 underflows)");
    // the largest reference tile (8 x 8 down to 1 x 1) whose region fits
    int t = 8;
    size_t bytes = 0;
    for (; t >= 1; t /= 2) {
        const int rows = std::min(H, (t - 1) * stride + 2 * Q.h + patch);
        const int cols = std::min(W, (t - 1) * stride + 2 * Q.h + patch);
        bytes = (size_t)rows * (cols * C + 15) * sizeof(float2);
        if (bytes <= (size_t)kNlmSmemLimit) break;
    }
    if (t < 1) return set_error(BM_ERR_UNSUPPORTED, "search region does not fit in shared memory");
    Q.ty = Q.tx = t;
    Q.tiles_x = (Q.n_rx + t - 1) / t;
    const int tiles = ((Q.n_ry + t - 1) / t) * Q.tiles_x;
    DevGuard dg(ctx_device(ctx));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) {
        kern<<<tiles, kNlmThreads, bytes, reinterpret_cast<cudaStream_t>(stream)>>>(Q);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("nlm launch: ") + cudaGetErrorString(e)).c_str());
    return BM_OK;
}

}  // extern "C"
