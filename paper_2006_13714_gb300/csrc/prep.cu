// prep.cu -- (a1) patch-norm box filter, the centring offset and the bf16
// operand planes; every kernel takes a table of jobs (one launch per stage
// for a whole batch of images).
//
// The box filter is the h_X (.) h_X vector of §III-B: the squared norm of
// every candidate patch, a p x p (x C) box sum of the squared image
// (Lemma 2 uses it as the ||X_j||^2 term; the same array read at a
// reference gives ||X_r||^2).  It is HBM-bound: one pass over the image,
// one write of the (H-p+1) x (W-p+1) result (plus its split copy for the
// tensor-core norm K-step).
#include "bm_internal.h"

#include <algorithm>
#include <cuda_bf16.h>

namespace bm {
namespace {

// Distances are shift-invariant, so the operands are centred before the
// split: uint8 by the exact constant 128, float32 by a sampled image mean.
// Smaller magnitudes shrink ||X_r||^2 + ||X_j||^2, which bounds the error of
// the split-precision cross term.
constexpr int kCenterU8 = 128;
constexpr int kMaxPrepJobs = 64;

struct PrepParams {
    int n;
    PrepJob jobs[kMaxPrepJobs];
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
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

// ---------------------------------------------------------------- centre
// Sampled mean of a float32 image: every step-th element (step = n / 2^14
// for large images), compensated FP32 sums, fixed order (each thread its
// samples in increasing order, then a fixed pairwise tree), so the value is
// deterministic.  One block per job; uint8 jobs use the constant 128.
constexpr int kCenterThreads = 512;

__global__ void __launch_bounds__(kCenterThreads) center_kernel(const __grid_constant__ PrepParams P) {
    const PrepJob& J = P.jobs[blockIdx.x];
    if (threadIdx.x == 0 && J.status) *J.status = 0;
    if (J.dtype != kF32 || J.ncc) {
        if (threadIdx.x == 0) *J.center = 0.f;  // uint8: constant offset, nothing to compute
        return;
    }
    __shared__ float2 part[kCenterThreads];
    __shared__ unsigned cnts[kCenterThreads];
    const float* img = static_cast<const float*>(J.img);
    const size_t n = (size_t)J.H * J.W * J.C;
    const size_t step = n > (1u << 14) ? n >> 14 : 1;
    const size_t count = (n + step - 1) / step;
    Acc2 acc{0.f, 0.f};
    unsigned cnt = 0;
    for (size_t j0 = threadIdx.x; j0 < count; j0 += (size_t)kCenterThreads * 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const size_t j = j0 + (size_t)k * kCenterThreads;
            v[k] = j < count ? __ldg(img + j * step) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (j0 + (size_t)k * kCenterThreads < count) {
                acc.add(v[k]);
                ++cnt;
            }
        }
    }
    part[threadIdx.x] = make_float2(acc.hi, acc.lo);
    cnts[threadIdx.x] = cnt;
    __syncthreads();
    for (int half = kCenterThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half) {
            const float2 a = part[threadIdx.x], b = part[threadIdx.x + half];
            Acc2 s{a.x, a.y};
            s.add(b.x);
            s.lo += b.y;
            part[threadIdx.x] = make_float2(s.hi, s.lo);
            cnts[threadIdx.x] += cnts[threadIdx.x + half];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned c = cnts[0];
        *J.center = c ? (part[0].x + part[0].y) / (float)c : 0.f;
    }
}

// ---------------------------------------------------------------- planes
// bf16 planes: plane row y holds W pixels of Cp channels (zero channel
// padding), then zero columns up to the pitch; rows >= H are zero.
// Grid (blocks per job, jobs); each block strides over its job.
template <bool kIsU8>
__global__ void planes_kernel(const __grid_constant__ PrepParams P) {
    const PrepJob& J = P.jobs[blockIdx.y];
    if ((J.dtype == (int)DType::kU8) != kIsU8) return;
    const float c0 = J.ncc ? 0.f : kIsU8 ? (float)kCenterU8 : *J.center;
    const bool two = !kIsU8 || J.ncc;  // a lo plane (zero for uint8: exact in bf16)
    const int vec_per_row = J.plane_pitch / 8;
    const size_t total = (size_t)J.plane_rows * vec_per_row;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(t / vec_per_row);
        const int e0 = (int)(t % vec_per_row) * 8;
        uint16_t hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = e0 + i;
            const int x = e / J.Cp, c = e % J.Cp;
            float v = 0.f;
            if (y < J.H && x < J.W && c < J.C) {
                size_t src = ((size_t)y * J.W + x) * J.C + c;
                v = (kIsU8 ? (float)static_cast<const uint8_t*>(J.img)[src]
                         : static_cast<const float*>(J.img)[src]) - c0;
            }
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[i] = __bfloat16_as_ushort(h);
            lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
        }
        uint4 vh, vl;
        vh.x = hi[0] | (uint32_t(hi[1]) << 16);
        vh.y = hi[2] | (uint32_t(hi[3]) << 16);
        vh.z = hi[4] | (uint32_t(hi[5]) << 16);
        vh.w = hi[6] | (uint32_t(hi[7]) << 16);
        reinterpret_cast<uint4*>(J.plane0)[t] = vh;
        if (two) {
            vl.x = lo[0] | (uint32_t(lo[1]) << 16);
            vl.y = lo[2] | (uint32_t(lo[3]) << 16);
            vl.z = lo[4] | (uint32_t(lo[5]) << 16);
            vl.w = lo[6] | (uint32_t(lo[7]) << 16);
            reinterpret_cast<uint4*>(J.plane1)[t] = vl;
        }
    }
}

// ---------------------------------------------------------------- box filter
// One block per output tile of kBoxR rows x kBoxX columns of one job.
//   1. hs[r][c] = sum over the p*C elements of input row y0 + r starting at
//      pixel x0 + c of (x - c0)^2 (integer for uint8; compensated hi/lo
//      for float32, element order e = 0 .. p*C-1);
//   2. out[r][c] = sum_{u < p} hs[r + u][c] in order u = 0 .. p-1;
//   3. nrm written row-major, nsp (split pieces) column-major, both with
//      consecutive threads on consecutive addresses.
// The arithmetic order is the same for every output, so the result is
// deterministic and independent of the tiling.
constexpr int kBoxThreads = 256;
constexpr int kBoxR = 32;
constexpr int kBoxX = 64;
constexpr int kBoxInRows = kBoxR + 15;  // p <= 16

template <bool kIsU8>
__global__ void __launch_bounds__(kBoxThreads) box_kernel(const __grid_constant__ PrepParams P) {
    const PrepJob& J = P.jobs[blockIdx.z];
    if ((J.dtype == (int)DType::kU8) != kIsU8) return;
    const int x0 = blockIdx.x * kBoxX, y0 = blockIdx.y * kBoxR;
    if (x0 >= J.Wc || y0 >= J.Hc) return;
    __shared__ float2 hs[kBoxInRows * kBoxX];
    __shared__ float outs[kBoxR * kBoxX];
    const int p = J.p, C = J.C, pc = p * C;
    const int orows = min(kBoxR, J.Hc - y0), ocols = min(kBoxX, J.Wc - x0);
    const int irows = orows + p - 1;
    const float c0 = kIsU8 ? 0.f : *J.center;
    // 1. horizontal sums of squares
    for (int idx = threadIdx.x; idx < irows * kBoxX; idx += kBoxThreads) {
        const int r = idx / kBoxX, c = idx % kBoxX;
        if (c >= ocols) continue;
        const size_t base = ((size_t)(y0 + r) * J.W + (x0 + c)) * C;
        if (kIsU8) {
            const uint8_t* row = static_cast<const uint8_t*>(J.img) + base;
            const int cu = J.ncc ? 0 : kCenterU8;
            int rs = 0;
            for (int e = 0; e < pc; ++e) {
                const int v = (int)__ldg(row + e) - cu;
                rs += v * v;
            }
            hs[idx] = make_float2(__int_as_float(rs), 0.f);
        } else {
            const float* row = static_cast<const float*>(J.img) + base;
            Acc2 a{0.f, 0.f};
            for (int e = 0; e < pc; ++e) {
                const float v = __ldg(row + e) - c0;
                const float sq = v * v;
                const float err = fmaf(v, v, -sq);  // exact square = sq + err
                a.add(sq);
                a.lo += err;
            }
            hs[idx] = make_float2(a.hi, a.lo);
        }
    }
    __syncthreads();
    // 2. vertical sums over p rows
    for (int idx = threadIdx.x; idx < kBoxR * kBoxX; idx += kBoxThreads) {
        const int r = idx / kBoxX, c = idx % kBoxX;
        if (r >= orows || c >= ocols) continue;
        if (kIsU8) {
            int sum = 0;
            for (int u = 0; u < p; ++u) sum += __float_as_int(hs[(r + u) * kBoxX + c].x);
            outs[idx] = __int_as_float(sum);
        } else {
            Acc2 s{0.f, 0.f};
            for (int u = 0; u < p; ++u) {
                const float2 h = hs[(r + u) * kBoxX + c];
                s.add(h.x);
                s.lo += h.y;
            }
            outs[idx] = s.hi + s.lo;
        }
    }
    __syncthreads();
    // 3. row-major norms (x fastest) ...
    for (int idx = threadIdx.x; idx < kBoxR * kBoxX; idx += kBoxThreads) {
        const int r = idx / kBoxX, c = idx % kBoxX;
        if (r >= orows || c >= ocols) continue;
        const size_t o = (size_t)(y0 + r) * J.Wc + (x0 + c);
        if (kIsU8) static_cast<int*>(J.nrm)[o] = __float_as_int(outs[idx]);
        else static_cast<float*>(J.nrm)[o] = outs[idx];
    }
    // ... and the column-major split copy (y fastest)
    if (J.nsp) {
        uint4* nsp = reinterpret_cast<uint4*>(J.nsp);
        for (int idx = threadIdx.x; idx < kBoxR * kBoxX; idx += kBoxThreads) {
            const int r = idx % kBoxR, c = idx / kBoxR;
            if (r >= orows || c >= ocols) continue;
            const float o = outs[r * kBoxX + c];
            const float v = kIsU8 ? (float)__float_as_int(o) : o;
            nsp[(size_t)(x0 + c) * J.Hc + (y0 + r)] =
                J.ncc ? make_uint4(__float_as_uint(v > 0.f ? rsqrtf(v) : 0.f), 0u, 0u, 0u)
                      : split_norm(v, !kIsU8);
        }
    }
}

template <class F>
cudaError_t for_chunks(const PrepJob* jobs, int n, F&& launch) {
    for (int i = 0; i < n; i += kMaxPrepJobs) {
        static thread_local PrepParams P;
        P.n = n - i < kMaxPrepJobs ? n - i : kMaxPrepJobs;
        for (int j = 0; j < P.n; ++j) P.jobs[j] = jobs[i + j];
        cudaError_t e = launch(P);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_center_batch(const PrepJob* jobs, int n, cudaStream_t st) {
    return for_chunks(jobs, n, [&](const PrepParams& P) {
        center_kernel<<<P.n, kCenterThreads, 0, st>>>(P);
        return cudaGetLastError();
    });
}

cudaError_t launch_planes_batch(const PrepJob* jobs, int n, cudaStream_t st) {
    return for_chunks(jobs, n, [&](const PrepParams& P) {
        size_t most = 0;
        bool u8 = false, f32 = false;
        for (int j = 0; j < P.n; ++j) {
            most = std::max(most, (size_t)P.jobs[j].plane_rows * (P.jobs[j].plane_pitch / 8));
            if (P.jobs[j].dtype == kU8) u8 = true;
            else f32 = true;
        }
        int bx = (int)((most + 255) / 256);
        if (bx > 64) bx = 64;
        if (bx < 1) bx = 1;
        dim3 grid(bx, P.n);
        if (u8) planes_kernel<true><<<grid, 256, 0, st>>>(P);
        if (f32) planes_kernel<false><<<grid, 256, 0, st>>>(P);
        return cudaGetLastError();
    });
}

cudaError_t launch_box_batch(const PrepJob* jobs, int n, cudaStream_t st) {
    return for_chunks(jobs, n, [&](const PrepParams& P) {
        int mx = 1, my = 1;
        bool u8 = false, f32 = false;
        for (int j = 0; j < P.n; ++j) {
            mx = std::max(mx, (P.jobs[j].Wc + kBoxX - 1) / kBoxX);
            my = std::max(my, (P.jobs[j].Hc + kBoxR - 1) / kBoxR);
            if (P.jobs[j].dtype == kU8) u8 = true;
            else f32 = true;
        }
        dim3 grid(mx, my, P.n);
        if (u8) box_kernel<true><<<grid, kBoxThreads, 0, st>>>(P);
        if (f32) box_kernel<false><<<grid, kBoxThreads, 0, st>>>(P);
        return cudaGetLastError();
    });
}

PrepJob make_prep_job(const Geom& g, const void* img, float* center, uint16_t* plane0,
                      uint16_t* plane1, void* nrm, uint16_t* nsp) {
    PrepJob j{};
    j.img = img; j.center = center; j.plane0 = plane0; j.plane1 = plane1; j.nrm = nrm; j.nsp = nsp;
    j.H = g.H; j.W = g.W; j.C = g.C; j.Cp = g.Cp; j.p = g.p; j.Hc = g.Hc; j.Wc = g.Wc;
    j.plane_pitch = g.plane_pitch; j.plane_rows = g.plane_rows; j.dtype = g.dtype;
    j.ncc = g.ncc;
    return j;
}

cudaError_t launch_center(const Geom& g, const void* img, float* center, cudaStream_t st) {
    const PrepJob j = make_prep_job(g, img, center, nullptr, nullptr, nullptr, nullptr);
    return launch_center_batch(&j, 1, st);
}

cudaError_t launch_boxfilter(const Geom& g, const void* img, const float* center, void* nrm,
                             uint16_t* nsp, cudaStream_t st) {
    const PrepJob j = make_prep_job(g, img, const_cast<float*>(center), nullptr, nullptr, nrm, nsp);
    return launch_box_batch(&j, 1, st);
}

cudaError_t launch_planes(const Geom& g, const void* img, const float* center, uint16_t* plane0,
                          uint16_t* plane1, cudaStream_t st) {
    const PrepJob j = make_prep_job(g, img, const_cast<float*>(center), plane0, plane1, nullptr, nullptr);
    return launch_planes_batch(&j, 1, st);
}

}  // namespace bm
