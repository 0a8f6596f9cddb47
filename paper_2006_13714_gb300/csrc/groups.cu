// groups.cu -- the steps on either side of block matching in the paper's
// restoration pipeline (§IV): patch-group formation and image
// reconstruction.
//
//   Group matrix (§IV, the equation after Eq. equ:self-convMM):
//     Y_r = [y_S(1), ..., y_S(K)], the K matched patches of reference r side
//     by side.  Stored as groups[r][k][(u*p + v)*C + c] =
//     X[y_k + u][x_k + v][c] with idx[r][k] = y_k*W + x_k; a missing match
//     (idx -1, or an index outside the candidate grid) is a zero patch.
//   Reconstruction (§IV, "Image Reconstruction"): every patch Z[r][k] of
//   every processed group is deposited back at idx[r][k] (summed), and each
//   pixel is divided by the number of deposited patches that contain it --
//   with weights w[r][k], by their sum: out = sum w Z / sum w.  Pixels no
//   patch covers are 0.
//
// GB300 layout of the work.  Gather: one thread per vector of a patch row
// (16-byte stores when the row length allows), indices checked against the
// candidate grid, the image read through L2.  Aggregate: one block per 8 x 8
// tile of the reference grid; the block accumulates its tile's K*64 patches
// into a shared-memory copy of their bounding box (shared atomics), then adds
// the box to the output with one global atomic per pixel and channel.  A
// block whose box does not fit in shared memory adds its patches to the
// output directly.  A last pass divides by the weight.
#include "bm.h"
#include "bm_internal.h"

#include <string>

namespace bm {
namespace {

constexpr int kAggTile = 8;                  // references per tile side
constexpr int kAggThreads = 256;
constexpr int kAggSmemBytes = 112 * 1024;     // bounding-box accumulator per block

__device__ __forceinline__ bool valid_top_left(int id, int H, int W, int p) {
    if (id < 0 || id >= H * W) return false;
    const int y = id / W, x = id - (id / W) * W;
    return y <= H - p && x <= W - p;
}

// ---------------------------------------------------------------- gather

template <typename T, int V>
struct VecOf;
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<uint8_t, 16> { using type = uint4; };
template <> struct VecOf<uint8_t, 8> { using type = uint2; };
template <> struct VecOf<uint8_t, 4> { using type = uint32_t; };
template <> struct VecOf<uint8_t, 1> { using type = uint8_t; };

// out[row][j] with row = (r*K + k)*p + u, j < p*C: the thread of vector
// (row, jv) writes elements jv*V .. jv*V + V - 1 of that row.
// I: index type (32-bit when the vector count allows: cheaper divisions).
template <typename T, int V, typename I>
__global__ void __launch_bounds__(256) gather_kernel(const T* __restrict__ img,
                                                     const int32_t* __restrict__ idx,
                                                     T* __restrict__ out, I n_vec, int H,
                                                     int W, int C, int p, int vec_per_row) {
    using Vec = typename VecOf<T, V>::type;
    const int rowlen = p * C;
    for (I e = (I)blockIdx.x * blockDim.x + threadIdx.x; e < n_vec; e += (I)gridDim.x * blockDim.x) {
        const I row = e / (I)vec_per_row;
        const int jv = (int)(e - row * (I)vec_per_row);
        const I patch = row / (I)p;
        const int u = (int)(row - patch * (I)p);
        const int id = __ldg(idx + patch);
        union {
            Vec v;
            T s[V];
        } buf;
        if (valid_top_left(id, H, W, p)) {
            const int y = id / W, x = id - (id / W) * W;
            const T* src = img + ((size_t)(y + u) * W + x) * C + jv * V;
#pragma unroll
            for (int i = 0; i < V; ++i) buf.s[i] = __ldg(src + i);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) buf.s[i] = T(0);
        }
        reinterpret_cast<Vec*>(out + (size_t)row * rowlen)[jv] = buf.v;
    }
}

template <typename T, int V>
cudaError_t launch_gather_t(const void* img, const int32_t* idx, void* out, long long n_rows,
                            int H, int W, int C, int p, cudaStream_t st) {
    const int vec_per_row = p * C / V;
    const long long n_vec = n_rows * vec_per_row;
    if (n_vec == 0) return cudaSuccess;
    long long blocks = (n_vec + 255) / 256;
    const long long cap = 152LL * 16;  // grid-stride beyond 16 blocks per SM
    if (blocks > cap) blocks = cap;
    if (n_vec < (1LL << 31))
        gather_kernel<T, V, unsigned><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const T*>(img), idx, static_cast<T*>(out), (unsigned)n_vec, H, W, C, p,
            vec_per_row);
    else
        gather_kernel<T, V, unsigned long long><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const T*>(img), idx, static_cast<T*>(out), (unsigned long long)n_vec, H,
            W, C, p, vec_per_row);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- aggregate

struct AggParams {
    const float* groups;   // [n_ry*n_rx][K][p*p*C]
    const int32_t* idx;    // [n_ry*n_rx][K]
    const float* weights;  // nullable, [n_ry*n_rx][K]
    float* out;            // [H][W][C] sums (zeroed before)
    float* wsum;           // [H][W] weights (zeroed before)
    int H, W, C, p, K, n_ry, n_rx, tiles_x;
    int smem_floats;       // capacity of the shared bounding-box accumulator
};

// Deposit one patch row (u) of patch `pt` of the tile: into the shared box
// (sbox != nullptr) or directly into the output.
__device__ __forceinline__ void deposit_row(const AggParams& P, long long pt, int u, int id,
                                            float* sbox, int by0, int bx0, int bw, int area) {
    const int C = P.C, p = P.p;
    const int y = id / P.W, x = id - (id / P.W) * P.W;
    const float w = P.weights ? __ldg(P.weights + pt) : 1.0f;
    const float* z = P.groups + ((size_t)pt * p + u) * (size_t)(p * C);
    if (sbox) {
        float* srow = sbox + ((y + u - by0) * bw + (x - bx0)) * C;
        float* wrow = sbox + (size_t)area * C + (y + u - by0) * bw + (x - bx0);
        for (int v = 0; v < p; ++v) {
            for (int c = 0; c < C; ++c) atomicAdd(srow + v * C + c, w * __ldg(z + v * C + c));
            atomicAdd(wrow + v, w);
        }
    } else {
        float* orow = P.out + ((size_t)(y + u) * P.W + x) * C;
        float* wrow = P.wsum + (size_t)(y + u) * P.W + x;
        for (int v = 0; v < p; ++v) {
            for (int c = 0; c < C; ++c) atomicAdd(orow + v * C + c, w * __ldg(z + v * C + c));
            atomicAdd(wrow + v, w);
        }
    }
}

// Tile patch t (reference row-major inside the tile, then k) -> global patch index.
__device__ __forceinline__ long long tile_patch(const AggParams& P, int t, int ry0, int rx0, int ntx) {
    const int k = t % P.K, rl = t / P.K;
    const int r = (ry0 + rl / ntx) * P.n_rx + rx0 + rl % ntx;
    return (long long)r * P.K + k;
}

__global__ void __launch_bounds__(kAggThreads) aggregate_kernel(const AggParams P) {
    extern __shared__ float sbox[];
    __shared__ int s_box[4];
    const int ty = blockIdx.x / P.tiles_x, tx = blockIdx.x - (blockIdx.x / P.tiles_x) * P.tiles_x;
    const int ry0 = ty * kAggTile, rx0 = tx * kAggTile;
    const int nty = min(kAggTile, P.n_ry - ry0), ntx = min(kAggTile, P.n_rx - rx0);
    const int npatch = nty * ntx * P.K;  // patches of the tile
    const int p = P.p, C = P.C;
    // (1) bounding box of the tile's valid patches
    int ymin = 1 << 30, xmin = 1 << 30, ymax = -1, xmax = -1;
    for (int t = threadIdx.x; t < npatch; t += blockDim.x) {
        const int id = __ldg(P.idx + tile_patch(P, t, ry0, rx0, ntx));
        if (!valid_top_left(id, P.H, P.W, p)) continue;
        const int y = id / P.W, x = id - (id / P.W) * P.W;
        ymin = min(ymin, y); ymax = max(ymax, y);
        xmin = min(xmin, x); xmax = max(xmax, x);
    }
    if (threadIdx.x == 0) {
        s_box[0] = 1 << 30; s_box[1] = 1 << 30; s_box[2] = -1; s_box[3] = -1;
    }
    __syncthreads();
    ymin = __reduce_min_sync(0xffffffffu, ymin);
    xmin = __reduce_min_sync(0xffffffffu, xmin);
    ymax = __reduce_max_sync(0xffffffffu, ymax);
    xmax = __reduce_max_sync(0xffffffffu, xmax);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_box[0], ymin); atomicMin(&s_box[1], xmin);
        atomicMax(&s_box[2], ymax); atomicMax(&s_box[3], xmax);
    }
    __syncthreads();
    if (s_box[2] < 0) return;  // no valid patch in this tile
    const int by0 = s_box[0], bx0 = s_box[1];
    const int bh = s_box[2] - by0 + p, bw = s_box[3] - bx0 + p;
    const int area = bh * bw;
    const bool use_smem = (long long)area * (C + 1) <= P.smem_floats;
    float* box = use_smem ? sbox : nullptr;
    if (use_smem) {
        for (int i = threadIdx.x; i < area * (C + 1); i += blockDim.x) sbox[i] = 0.f;
        __syncthreads();
    }
    // (2) deposit: one patch row per thread and step (consecutive threads read
    // consecutive rows of the groups array)
    for (int t = threadIdx.x; t < npatch * p; t += blockDim.x) {
        const int tp = t / p, u = t - tp * p;
        const long long pt = tile_patch(P, tp, ry0, rx0, ntx);
        const int id = __ldg(P.idx + pt);
        if (!valid_top_left(id, P.H, P.W, p)) continue;
        deposit_row(P, pt, u, id, box, by0, bx0, bw, area);
    }
    if (!use_smem) return;
    __syncthreads();
    // (3) add the box to the output (pixels some patch touched)
    for (int i = threadIdx.x; i < area; i += blockDim.x) {
        const float wv = sbox[(size_t)area * C + i];
        bool touched = wv != 0.f;
        for (int c = 0; c < C && !touched; ++c) touched = sbox[i * C + c] != 0.f;
        if (!touched) continue;
        const int yy = by0 + i / bw, xx = bx0 + i % bw;
        float* o = P.out + ((size_t)yy * P.W + xx) * C;
        for (int c = 0; c < C; ++c) atomicAdd(o + c, sbox[i * C + c]);
        atomicAdd(P.wsum + (size_t)yy * P.W + xx, wv);
    }
}

// out[y][x][c] /= wsum[y][x] (0 where the weight is 0).
__global__ void __launch_bounds__(256) normalize_kernel(float* __restrict__ out,
                                                        const float* __restrict__ wsum,
                                                        long long n_pix, int C) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_pix * C;
         i += (long long)gridDim.x * blockDim.x) {
        const float w = __ldg(wsum + i / C);
        out[i] = w != 0.f ? out[i] / w : 0.f;
    }
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

int check_common(const bm_ctx* ctx, int H, int W, int C, int patch, int n_ry, int n_rx, int K) {
    if (!ctx) return set_error(BM_ERR_INVALID, "null context");
    if (H < 1 || W < 1 || C < 1 || C > kMaxC || patch < 1 || patch > H || patch > W)
        return set_error(BM_ERR_INVALID, "invalid image or patch geometry");
    if (n_ry < 0 || n_rx < 0 || K < 1 || K > kMaxK)
        return set_error(BM_ERR_INVALID, "invalid reference grid or K");
    if ((long long)H * W >= (1LL << 31))
        return set_error(BM_ERR_UNSUPPORTED, "H*W must be below 2^31");
    return BM_OK;
}

}  // namespace

cudaError_t launch_gather_groups(const void* img, int dtype, const int32_t* idx, void* out,
                                 long long n_patches, int H, int W, int C, int p,
                                 cudaStream_t st) {
    const long long rows = n_patches * p;
    const int rowlen = p * C;
    const uintptr_t a = reinterpret_cast<uintptr_t>(out);
    if (dtype == kF32) {
        if (rowlen % 4 == 0 && a % 16 == 0) return launch_gather_t<float, 4>(img, idx, out, rows, H, W, C, p, st);
        if (rowlen % 2 == 0 && a % 8 == 0) return launch_gather_t<float, 2>(img, idx, out, rows, H, W, C, p, st);
        return launch_gather_t<float, 1>(img, idx, out, rows, H, W, C, p, st);
    }
    if (rowlen % 16 == 0 && a % 16 == 0) return launch_gather_t<uint8_t, 16>(img, idx, out, rows, H, W, C, p, st);
    if (rowlen % 8 == 0 && a % 8 == 0) return launch_gather_t<uint8_t, 8>(img, idx, out, rows, H, W, C, p, st);
    if (rowlen % 4 == 0 && a % 4 == 0) return launch_gather_t<uint8_t, 4>(img, idx, out, rows, H, W, C, p, st);
    return launch_gather_t<uint8_t, 1>(img, idx, out, rows, H, W, C, p, st);
}

cudaError_t launch_aggregate(const float* groups, const int32_t* idx, const float* weights,
                             int n_ry, int n_rx, int K, int H, int W, int C, int p, float* out,
                             float* wsum, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(out, 0, (size_t)H * W * C * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(wsum, 0, (size_t)H * W * sizeof(float), st)) != cudaSuccess) return e;
    const int tiles_y = (n_ry + kAggTile - 1) / kAggTile, tiles_x = (n_rx + kAggTile - 1) / kAggTile;
    if (tiles_y > 0 && tiles_x > 0) {
        AggParams P{groups, idx, weights, out, wsum, H, W, C, p, K, n_ry, n_rx, tiles_x,
                    kAggSmemBytes / (int)sizeof(float)};
        if ((e = cudaFuncSetAttribute(aggregate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kAggSmemBytes)) != cudaSuccess)
            return e;
        aggregate_kernel<<<tiles_y * tiles_x, kAggThreads, kAggSmemBytes, st>>>(P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const long long n = (long long)H * W * C;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    normalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(out, wsum, (long long)H * W, C);
    return cudaGetLastError();
}

}  // namespace bm

using namespace bm;

extern "C" {

int bm_gather_groups(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype,
                     int patch, const int32_t* idx, int n_ry, int n_rx, int K, void* out_groups,
                     bm_stream stream) {
    int rc = check_common(ctx, H, W, C, patch, n_ry, n_rx, K);
    if (rc != BM_OK) return rc;
    if (dtype != BM_U8 && dtype != BM_F32) return set_error(BM_ERR_INVALID, "unknown dtype");
    const long long n_patches = (long long)n_ry * n_rx * K;
    if (n_patches == 0) return BM_OK;
    if (!img || !idx || !out_groups) return set_error(BM_ERR_INVALID, "null pointer");
    DevGuard dg(ctx_device(ctx));
    const cudaError_t e = launch_gather_groups(img, dtype == BM_U8 ? kU8 : kF32, idx, out_groups,
                                               n_patches, H, W, C, patch,
                                               reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("gather launch: ") + cudaGetErrorString(e)).c_str());
    return BM_OK;
}

int bm_aggregate(bm_ctx* ctx, const float* groups, const int32_t* idx, const float* weights,
                 int n_ry, int n_rx, int K, int H, int W, int C, int patch, float* out_img,
                 float* out_weight, bm_stream stream) {
    int rc = check_common(ctx, H, W, C, patch, n_ry, n_rx, K);
    if (rc != BM_OK) return rc;
    const long long n_patches = (long long)n_ry * n_rx * K;
    if (!out_img || !out_weight || (n_patches > 0 && (!groups || !idx)))
        return set_error(BM_ERR_INVALID, "null pointer");
    DevGuard dg(ctx_device(ctx));
    const cudaError_t e = launch_aggregate(groups, idx, weights, n_ry, n_rx, K, H, W, C, patch,
                                           out_img, out_weight,
                                           reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("aggregate launch: ") + cudaGetErrorString(e)).c_str());
    return BM_OK;
}

}  // extern "C"
