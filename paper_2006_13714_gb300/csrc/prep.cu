// prep.cu -- (a1) patch-norm box filter and the bf16 operand planes.
//
// The box filter is the h_X (.) h_X vector of §III-B: the squared norm of
// every candidate patch, a p x p (x C) box sum of the squared image
// (Lemma 2 uses it as the ||X_j||^2 term; the same array read at a
// reference gives ||X_r||^2).  It is HBM-bound: one pass over the image,
// one write of the (H-p+1) x (W-p+1) result.
#include "bm_internal.h"

#include <cuda_bf16.h>

namespace bm {
namespace {

constexpr int kBoxThreads = 128;
// Distances are shift-invariant, so the operands are centred before the
// split: uint8 by the exact constant 128, float32 by a sampled image mean.
// Smaller magnitudes shrink ||X_r||^2 + ||X_j||^2, which bounds the error of
// the split-precision cross term.
constexpr int kCenterU8 = 128;
constexpr int kBoxRows = 32;  // output rows per block (strip)

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
// x = hi + mid + lo exactly for any float with <= 24 significant bits (the
// norm pieces of the tensor-core norm K-step).
__device__ __forceinline__ uint4 split_norm(float x, bool two_copies) {
    const uint16_t hi = bf16_bits(x);
    const float r1 = x - __bfloat162float(__ushort_as_bfloat16(hi));
    const uint16_t mid = bf16_bits(r1);
    const float r2 = r1 - __bfloat162float(__ushort_as_bfloat16(mid));
    const uint16_t lo = bf16_bits(r2);
    if (two_copies)
        return make_uint4(hi | (uint32_t(mid) << 16), lo | (uint32_t(hi) << 16),
                          mid | (uint32_t(lo) << 16), 0u);
    return make_uint4(hi | (uint32_t(mid) << 16), lo, 0u, 0u);
}

// Compensated accumulator: value = hi + lo to about one float ulp.
struct Acc2 {
    float hi, lo;
    __device__ __forceinline__ void add(float x) {
        float s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo += e;
    }
};

// One thread per output column; each block walks a strip of kBoxRows output
// rows.  The last p row sums live in a per-thread shared-memory ring so every
// image row is read once per column; output = sum of the p ring entries in
// fixed order (deterministic).  With nsp, each value is also written as its
// bf16 pieces, column-major (a column of a chunk is one contiguous copy).
template <bool kU8>
__global__ void __launch_bounds__(kBoxThreads)
boxfilter_kernel(const void* __restrict__ img, int W, int C, int p, int Hc, int Wc,
                 const float* __restrict__ center, void* __restrict__ nrm,
                 uint4* __restrict__ nsp) {
    extern __shared__ unsigned char smem_raw[];
    const int x = blockIdx.x * kBoxThreads + threadIdx.x;
    if (x >= Wc) return;
    const int y0 = blockIdx.y * kBoxRows;
    const int y1 = min(y0 + kBoxRows, Hc);
    const int row_elems = W * C;
    if (kU8) {
        int* ring = reinterpret_cast<int*>(smem_raw);
        const uint8_t* im = static_cast<const uint8_t*>(img);
        for (int y = y0; y < y1 + p - 1; ++y) {
            const uint8_t* row = im + (size_t)y * row_elems + (size_t)x * C;
            int rs = 0;
            for (int e = 0; e < p * C; ++e) {
                int v = (int)row[e] - kCenterU8;
                rs += v * v;
            }
            ring[(y % p) * kBoxThreads + threadIdx.x] = rs;
            int yo = y - (p - 1);
            if (yo >= y0) {
                int sum = 0;
                for (int u = 0; u < p; ++u) sum += ring[((yo + u) % p) * kBoxThreads + threadIdx.x];
                static_cast<int*>(nrm)[(size_t)yo * Wc + x] = sum;
                if (nsp) nsp[(size_t)x * Hc + yo] = split_norm((float)sum, false);
            }
        }
    } else {
        float2* ring = reinterpret_cast<float2*>(smem_raw);
        const float* im = static_cast<const float*>(img);
        const float c0 = *center;
        for (int y = y0; y < y1 + p - 1; ++y) {
            const float* row = im + (size_t)y * row_elems + (size_t)x * C;
            Acc2 a{0.f, 0.f};
            for (int e = 0; e < p * C; ++e) {
                float v = row[e] - c0;
                float sq = v * v;
                float err = fmaf(v, v, -sq);  // exact square = sq + err
                a.add(sq);
                a.lo += err;
            }
            ring[(y % p) * kBoxThreads + threadIdx.x] = make_float2(a.hi, a.lo);
            int yo = y - (p - 1);
            if (yo >= y0) {
                Acc2 s{0.f, 0.f};
                for (int u = 0; u < p; ++u) {
                    float2 r = ring[((yo + u) % p) * kBoxThreads + threadIdx.x];
                    s.add(r.x);
                    s.lo += r.y;
                }
                const float v = s.hi + s.lo;
                static_cast<float*>(nrm)[(size_t)yo * Wc + x] = v;
                if (nsp) nsp[(size_t)x * Hc + yo] = split_norm(v, true);
            }
        }
    }
}

// bf16 planes: plane row y holds W pixels of Cp channels (zero channel
// padding), then zero columns up to the pitch; rows >= H are zero.
template <bool kU8>
__global__ void planes_kernel(const void* __restrict__ img, int H, int W, int C, int Cp,
                              int pitch, int rows, const float* __restrict__ center,
                              uint16_t* __restrict__ p0, uint16_t* __restrict__ p1) {
    const float c0 = kU8 ? (float)kCenterU8 : *center;
    const int vec_per_row = pitch / 8;
    const size_t total = (size_t)rows * vec_per_row;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(t / vec_per_row);
        const int e0 = (int)(t % vec_per_row) * 8;
        uint16_t hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = e0 + i;
            const int x = e / Cp, c = e % Cp;
            float v = 0.f;
            if (y < H && x < W && c < C) {
                size_t src = ((size_t)y * W + x) * C + c;
                v = (kU8 ? (float)static_cast<const uint8_t*>(img)[src]
                         : static_cast<const float*>(img)[src]) - c0;
            }
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[i] = __bfloat16_as_ushort(h);
            if (!kU8) lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
        }
        uint4 vh, vl;
        vh.x = hi[0] | (uint32_t(hi[1]) << 16);
        vh.y = hi[2] | (uint32_t(hi[3]) << 16);
        vh.z = hi[4] | (uint32_t(hi[5]) << 16);
        vh.w = hi[6] | (uint32_t(hi[7]) << 16);
        reinterpret_cast<uint4*>(p0)[t] = vh;
        if (!kU8) {
            vl.x = lo[0] | (uint32_t(lo[1]) << 16);
            vl.y = lo[2] | (uint32_t(lo[3]) << 16);
            vl.z = lo[4] | (uint32_t(lo[5]) << 16);
            vl.w = lo[6] | (uint32_t(lo[7]) << 16);
            reinterpret_cast<uint4*>(p1)[t] = vl;
        }
    }
}

// Sampled mean of a float32 image (one block, fixed summation order, so the
// value is deterministic; compensated FP32 sums -- FP64 is slow on this
// part); uint8 uses the constant 128.
__global__ void __launch_bounds__(256) center_kernel(const float* __restrict__ img, size_t n,
                                                     float* __restrict__ center) {
    __shared__ float2 part[256];
    __shared__ unsigned cnts[256];
    const size_t step = n > (1u << 14) ? n >> 14 : 1;
    Acc2 acc{0.f, 0.f};
    unsigned cnt = 0;
    for (size_t i = threadIdx.x * step; i < n; i += 256 * step) {
        acc.add(img[i]);
        ++cnt;
    }
    part[threadIdx.x] = make_float2(acc.hi, acc.lo);
    cnts[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc2 s{0.f, 0.f};
        unsigned c = 0;
        for (int t = 0; t < 256; ++t) {
            s.add(part[t].x);
            s.lo += part[t].y;
            c += cnts[t];
        }
        *center = c ? (s.hi + s.lo) / (float)c : 0.f;
    }
}

}  // namespace

cudaError_t launch_center(const Geom& g, const void* img, float* center, cudaStream_t st) {
    if (g.dtype == kU8) {
        // constant; nothing to compute
        return cudaMemsetAsync(center, 0, sizeof(float), st);
    }
    center_kernel<<<1, 256, 0, st>>>(static_cast<const float*>(img), (size_t)g.H * g.W * g.C,
                                     center);
    return cudaGetLastError();
}

cudaError_t launch_boxfilter(const Geom& g, const void* img, const float* center, void* nrm,
                             uint16_t* nsp, cudaStream_t st) {
    dim3 grid((g.Wc + kBoxThreads - 1) / kBoxThreads, (g.Hc + kBoxRows - 1) / kBoxRows);
    if (g.dtype == kU8) {
        size_t sm = (size_t)g.p * kBoxThreads * sizeof(int);
        boxfilter_kernel<true><<<grid, kBoxThreads, sm, st>>>(img, g.W, g.C, g.p, g.Hc, g.Wc, center, nrm,
                                                              reinterpret_cast<uint4*>(nsp));
    } else {
        size_t sm = (size_t)g.p * kBoxThreads * sizeof(float2);
        boxfilter_kernel<false><<<grid, kBoxThreads, sm, st>>>(img, g.W, g.C, g.p, g.Hc, g.Wc, center, nrm,
                                                              reinterpret_cast<uint4*>(nsp));
    }
    return cudaGetLastError();
}

cudaError_t launch_planes(const Geom& g, const void* img, const float* center, uint16_t* plane0,
                          uint16_t* plane1, cudaStream_t st) {
    size_t total = (size_t)g.plane_rows * (g.plane_pitch / 8);
    int threads = 256;
    int blocks = (int)((total + threads - 1) / threads);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (g.dtype == kU8)
        planes_kernel<true><<<blocks, threads, 0, st>>>(img, g.H, g.W, g.C, g.Cp, g.plane_pitch,
                                                        g.plane_rows, center, plane0, plane1);
    else
        planes_kernel<false><<<blocks, threads, 0, st>>>(img, g.H, g.W, g.C, g.Cp, g.plane_pitch,
                                                         g.plane_rows, center, plane0, plane1);
    return cudaGetLastError();
}

}  // namespace bm
