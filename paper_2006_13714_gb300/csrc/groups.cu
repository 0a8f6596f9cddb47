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
// GB300 layout of the work.
//   Gather: one block per 8 x 8 tile of the reference grid, i.e. per the
//   tile's 64*K patches, whose top-left corners lie in a small bounding box
//   (the union of the tile's search windows when the indices come from
//   bm_match).  The box of the image is staged in shared memory with
//   coalesced loads; the groups are then written with 16-byte streaming
//   stores in output order (a tile row of references is one contiguous
//   range).  A tile whose box does not fit reads the image directly.
//   Aggregate: the weight map is a p x p box filter of a histogram of the
//   weights over top-left corners (one reduction per patch).  The sums: one
//   warp per patch, every lane busy; each patch row is added to the output
//   as the 4-pixel quads it overlaps with 16-byte vector reductions in L2
//   (zero outside the patch) -- about 22 reductions per 8 x 8 patch instead
//   of 128 scalar ones.  Shapes without aligned quads use scalar reductions.
//   A last pass divides by the weight.
#include "bm.h"
#include "bm_internal.h"

#include <string>

namespace bm {
namespace {

constexpr int kTile = 8;                   // references per tile side
constexpr int kThreads = 256;
constexpr int kChunk = 256;                // patches whose metadata is staged at a time
// Shared memory per block, sized so that every block of a 512 x 512 image
// (22 x 22 tiles) is resident at once (5 blocks / SM).
constexpr int kGatherSmem = 40 * 1024;     // image box (gather)
constexpr int kItems = 4;                  // aggregate: quad items per lane in flight

// Per-patch data of a chunk of a tile, staged in shared memory.
struct PatchMeta {
    int yrel;    // top-left row minus the box's first row (< 0: invalid)
    int xrel;    // top-left column minus the box's first column
    int pt;      // global patch index (r*K + k)
    float w;     // weight (aggregate)
};

struct TileParams {
    const void* img;       // gather: H x W x C image (uint8 / float32)
    void* groups;          // gather: output; aggregate: input (float32)
    const int32_t* idx;    // [n_ry*n_rx][K]
    const float* weights;  // aggregate, nullable
    float* out;            // aggregate: [H][W][C] sums (zeroed before)
    float* wsum;           // aggregate: [H][W] weights (zeroed before)
    int H, W, C, p, K, n_ry, n_rx, tiles_x;
    int plen;              // p*p*C
    bool vec;              // 16-byte vectors possible (alignment and lengths)
    FastDiv d_W, d_rowlen, d_vpp, d_plen;
};

struct Tile {
    int ry0, rx0, ntx, npatch;
};

__device__ __forceinline__ Tile tile_of(const TileParams& P) {
    Tile t;
    const int ty = blockIdx.x / P.tiles_x;
    const int tx = blockIdx.x - ty * P.tiles_x;
    t.ry0 = ty * kTile;
    t.rx0 = tx * kTile;
    const int nty = min(kTile, P.n_ry - t.ry0);
    t.ntx = min(kTile, P.n_rx - t.rx0);
    t.npatch = nty * t.ntx * P.K;
    return t;
}

// Tile patch i (reference row-major inside the tile, then k) -> global patch index.
__device__ __forceinline__ int tile_patch(const TileParams& P, const Tile& T, int i) {
    const int k = i % P.K, rl = i / P.K;
    const int r = (T.ry0 + rl / T.ntx) * P.n_rx + T.rx0 + rl % T.ntx;
    return r * P.K + k;
}

__device__ __forceinline__ bool top_left(const TileParams& P, int id, int& y, int& x) {
    if (id < 0 || id >= P.H * P.W) return false;
    y = fast_div(id, P.d_W);
    x = id - y * P.W;
    return y <= P.H - P.p && x <= P.W - P.p;
}

// Block-wide bounding box of the tile's valid top-left corners, extended by
// the patch: rows [by0, by0 + bh), columns [bx0, bx0 + bw); false if no
// patch is valid.  align4: the box starts and ends on 4-pixel boundaries.
__device__ bool tile_box(const TileParams& P, const Tile& T, bool align4, int& by0, int& bx0,
                         int& bh, int& bw) {
    __shared__ int s_box[4];
    int ymin = 1 << 30, xmin = 1 << 30, ymax = -1, xmax = -1;
    for (int i = threadIdx.x; i < T.npatch; i += blockDim.x) {
        int y, x;
        if (!top_left(P, __ldg(P.idx + tile_patch(P, T, i)), y, x)) continue;
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
    if (s_box[2] < 0) return false;
    by0 = s_box[0];
    bx0 = align4 ? (s_box[1] & ~3) : s_box[1];
    bh = s_box[2] - by0 + P.p;
    bw = s_box[3] - bx0 + P.p;
    if (align4) bw = (bw + 3) & ~3;  // stays inside the row: W % 4 == 0
    return true;
}

// Metadata of tile patches [c0, c0 + n) into s_meta (one thread per patch).
__device__ __forceinline__ void stage_meta(const TileParams& P, const Tile& T, int c0, int n,
                                           int by0, int bx0, PatchMeta* s_meta) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int pt = tile_patch(P, T, c0 + i);
        int y, x;
        PatchMeta m;
        m.pt = pt;
        m.w = P.weights ? __ldg(P.weights + pt) : 1.0f;
        if (top_left(P, __ldg(P.idx + pt), y, x)) {
            m.yrel = y - by0;
            m.xrel = x - bx0;
        } else {
            m.yrel = -(1 << 20);
            m.xrel = 0;
        }
        s_meta[i] = m;
    }
}

// ---------------------------------------------------------------- gather

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<uint8_t> { using type = uint4; static constexpr int n = 16; };

template <typename T>
__global__ void __launch_bounds__(kThreads) gather_kernel(const TileParams P) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ PatchMeta s_meta[kChunk];
    using V16 = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    T* sbox = reinterpret_cast<T*>(smem_raw);
    const T* img = static_cast<const T*>(P.img);
    T* out = static_cast<T*>(P.groups);
    const Tile Tl = tile_of(P);
    const int C = P.C, rowlen = P.p * C, plen = P.plen;
    int by0 = 0, bx0 = 0, bh = 0, bw = 0;
    const bool any = tile_box(P, Tl, false, by0, bx0, bh, bw);
    const bool staged = any && (long long)bh * bw * C * (int)sizeof(T) <= kGatherSmem;
    if (staged) {
        // the box, row by row (each row segment is contiguous in the image)
        const int seg = bw * C;
        for (int i = threadIdx.x; i < bh * seg; i += blockDim.x) {
            const int r = i / seg, j = i - r * seg;
            sbox[i] = __ldg(img + ((size_t)(by0 + r) * P.W + bx0) * C + j);
        }
    }
    const int spitch = bw * C;
    for (int c0 = 0; c0 < Tl.npatch; c0 += kChunk) {
        const int nc = min(kChunk, Tl.npatch - c0);
        __syncthreads();  // box staged / previous chunk's metadata consumed
        stage_meta(P, Tl, c0, nc, by0, bx0, s_meta);
        __syncthreads();
        const int vn = P.vec ? VN : 1;
        const int vpp = plen / vn;  // vectors per patch
        if (staged && P.vec && rowlen % VN == 0 && kThreads % vpp == 0) {
            // a vector stays inside a patch row, and each thread keeps its
            // place in a patch (row u, vector jv) for the whole loop
            const int vpr = rowlen / VN, pstep = kThreads / vpp;
            const int lt = threadIdx.x % vpp, u = lt / vpr, jv = lt - u * vpr;
            const int soff = u * spitch + jv * VN, goff = u * rowlen + jv * VN;
            for (int t = threadIdx.x / vpp; t < nc; t += pstep) {
                const PatchMeta m = s_meta[t];
                union {
                    V16 v;
                    T s[VN];
                } buf;
                const T* src = sbox + m.yrel * spitch + m.xrel * C + soff;
#pragma unroll
                for (int q = 0; q < VN; ++q) buf.s[q] = m.yrel >= 0 ? src[q] : T(0);
                __stcs(reinterpret_cast<V16*>(out + (size_t)m.pt * plen + goff), buf.v);
            }
            continue;
        }
        for (int i = threadIdx.x; i < nc * vpp; i += blockDim.x) {
            const int t = fast_div(i, P.vec ? P.d_vpp : P.d_plen), e0 = (i - t * vpp) * vn;
            const PatchMeta m = s_meta[t];
            union {
                V16 v;
                T s[VN];
            } buf;
#pragma unroll
            for (int q = 0; q < VN; ++q) {
                buf.s[q] = T(0);
                if (q < vn && m.yrel >= 0) {
                    const int e = e0 + q;
                    const int u = fast_div(e, P.d_rowlen), rem = e - u * rowlen;
                    buf.s[q] = staged ? sbox[(m.yrel + u) * spitch + m.xrel * C + rem]
                                      : __ldg(img + ((size_t)(by0 + m.yrel + u) * P.W + bx0 + m.xrel) * C + rem);
                }
            }
            T* dst = out + (size_t)m.pt * plen + e0;
            if (P.vec) __stcs(reinterpret_cast<V16*>(dst), buf.v);
            else *dst = buf.s[0];
        }
    }
}

// ---------------------------------------------------------------- aggregate

// Add 4 consecutive floats (16-byte aligned) to global memory in one reduction.
__device__ __forceinline__ void red4(float* dst, float4 v) {
    atomicAdd(reinterpret_cast<float4*>(dst), v);
}

// Sums: one warp per patch (grid-stride over all n_ry*n_rx*K patches), every
// lane busy.  vec (W % 4 == 0, 16-byte aligned buffers, C in {1, 4}): one
// channel -- a patch row is added as the 4-pixel quads it overlaps, zero
// outside the patch, one 16-byte reduction per quad; four channels -- one
// 16-byte reduction per pixel.  Otherwise one scalar reduction per element.
__global__ void __launch_bounds__(kThreads) aggregate_kernel(const TileParams P) {
    const int p = P.p, C = P.C, pC = p * C, plen = P.plen;
    const int lane = threadIdx.x & 31;
    const float* Z = static_cast<const float*>(P.groups);
    const long long n_patch = (long long)P.n_ry * P.n_rx * P.K;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    if (P.vec && C == 1) {
        // items (patch, row u, quad j) of a batch of patches, up to kItems per
        // lane, all loads issued before any reduction
        const int qmax = (p + 6) / 4;  // quads a patch row can overlap
        const int ipp = p * qmax;      // items per patch
        const int batch = max(1, 32 * kItems / ipp);
        for (long long b0 = warp0 * batch; b0 < n_patch; b0 += nwarps * batch) {
            float zv[kItems][4];
            long long gq[kItems];
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                gq[k] = -1;
                const int it = lane + 32 * k;
                if (it >= batch * ipp) continue;
                const int ps = it / ipp, rem = it - ps * ipp;
                const long long pt = b0 + ps;
                if (pt >= n_patch) continue;
                int y, x;
                if (!top_left(P, __ldg(P.idx + pt), y, x)) continue;
                const int u = rem / qmax, j = rem - u * qmax;
                const int v0 = 4 * j - (x & 3);  // patch column of the quad's first pixel
                if (v0 >= p) continue;           // quad past the patch row
                const float w = P.weights ? __ldg(P.weights + pt) : 1.0f;
                const float* z = Z + (size_t)pt * plen + u * p;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    zv[k][i] = (v0 + i >= 0 && v0 + i < p) ? w * __ldcs(z + v0 + i) : 0.f;
                gq[k] = (long long)(y + u) * P.W + (x & ~3) + 4 * j;
            }
#pragma unroll
            for (int k = 0; k < kItems; ++k)
                if (gq[k] >= 0) red4(P.out + gq[k], make_float4(zv[k][0], zv[k][1], zv[k][2], zv[k][3]));
        }
        return;
    }
    for (long long pt = warp0; pt < n_patch; pt += nwarps) {
        int y, x;
        if (!top_left(P, __ldg(P.idx + pt), y, x)) continue;
        const float w = P.weights ? __ldg(P.weights + pt) : 1.0f;
        const float* z = Z + (size_t)pt * plen;
        if (P.vec) {  // four channels: one 16-byte reduction per pixel
            for (int e = lane; e < p * p; e += 32) {
                const int u = e / p, v = e - u * p;
                float4 zz = __ldcs(reinterpret_cast<const float4*>(z) + e);
                zz.x *= w; zz.y *= w; zz.z *= w; zz.w *= w;
                red4(P.out + ((size_t)(y + u) * P.W + x + v) * 4, zz);
            }
        } else {
            for (int e = lane; e < plen; e += 32) {
                const int u = fast_div(e, P.d_rowlen), rem = e - u * pC;
                atomicAdd(P.out + ((size_t)(y + u) * P.W + x) * C + rem, w * __ldcs(z + e));
            }
        }
    }
}

// Weight histogram over top-left corners: hist[y][x] += w for every valid
// patch at (y, x).  hist is the first H*W floats of the (zeroed) output image.
__global__ void __launch_bounds__(kThreads) weight_hist_kernel(const TileParams P, float* hist) {
    const long long n_patch = (long long)P.n_ry * P.n_rx * P.K;
    for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < n_patch;
         pt += (long long)gridDim.x * blockDim.x) {
        int y, x;
        if (!top_left(P, __ldg(P.idx + pt), y, x)) continue;
        atomicAdd(hist + (size_t)y * P.W + x, P.weights ? __ldg(P.weights + pt) : 1.0f);
    }
}

// wsum[y][x] = sum_{u, v < p} hist[y - u][x - v] (the weight of every patch
// covering the pixel), separably over a 32 x 32 tile plus its halo in shared
// memory: row sums of p, then column sums of p.
constexpr int kBoxTile = 32;
__global__ void __launch_bounds__(kBoxTile * 8) weight_box_kernel(const float* __restrict__ hist,
                                                                 float* __restrict__ wsum, int H,
                                                                 int W, int p) {
    __shared__ float sh[kBoxTile + 16][kBoxTile + 16];   // halo p - 1 <= 15
    __shared__ float rs[kBoxTile + 16][kBoxTile];
    const int ty0 = blockIdx.y * kBoxTile, tx0 = blockIdx.x * kBoxTile;
    const int nh = kBoxTile + p - 1;
    for (int i = threadIdx.x; i < nh * nh; i += blockDim.x) {
        const int r = i / nh, c = i - r * nh;
        const int y = ty0 - (p - 1) + r, x = tx0 - (p - 1) + c;
        sh[r][c] = (y >= 0 && y < H && x >= 0 && x < W) ? hist[(size_t)y * W + x] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nh * kBoxTile; i += blockDim.x) {
        const int r = i / kBoxTile, c = i - r * kBoxTile;
        float a = 0.f;
        for (int v = 0; v < p; ++v) a += sh[r][c + v];
        rs[r][c] = a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBoxTile * kBoxTile; i += blockDim.x) {
        const int r = i / kBoxTile, c = i - r * kBoxTile;
        const int y = ty0 + r, x = tx0 + c;
        if (y >= H || x >= W) continue;
        float a = 0.f;
        for (int u = 0; u < p; ++u) a += rs[r + u][c];
        wsum[(size_t)y * W + x] = a;
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

TileParams make_params(const void* img, void* groups, const int32_t* idx, const float* weights,
                       float* out, float* wsum, int n_ry, int n_rx, int K, int H, int W, int C,
                       int p, bool vec, int vn) {
    TileParams P{};
    P.img = img; P.groups = groups; P.idx = idx; P.weights = weights; P.out = out; P.wsum = wsum;
    P.H = H; P.W = W; P.C = C; P.p = p; P.K = K; P.n_ry = n_ry; P.n_rx = n_rx;
    P.tiles_x = (n_rx + kTile - 1) / kTile;
    P.plen = p * p * C;
    P.vec = vec;
    P.d_W = make_fastdiv((unsigned)W);
    P.d_rowlen = make_fastdiv((unsigned)(p * C));
    P.d_vpp = make_fastdiv((unsigned)(vec ? P.plen / vn : 1));
    P.d_plen = make_fastdiv((unsigned)P.plen);
    return P;
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
    if (patch * patch * C > kMaxPatchElems)
        return set_error(BM_ERR_UNSUPPORTED, "patch*patch*C must be at most 256");
    if ((long long)n_ry * n_rx * K >= (1LL << 31))
        return set_error(BM_ERR_UNSUPPORTED, "n_ry*n_rx*K must be below 2^31");
    return BM_OK;
}

}  // namespace

cudaError_t launch_gather_groups(const void* img, int dtype, const int32_t* idx, void* out,
                                 int n_ry, int n_rx, int K, int H, int W, int C, int p,
                                 cudaStream_t st) {
    const int tiles = ((n_ry + kTile - 1) / kTile) * ((n_rx + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    const int esize = dtype == kF32 ? 4 : 1;
    const bool vec = (p * p * C * esize) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0;
    const TileParams P = make_params(img, out, idx, nullptr, nullptr, nullptr, n_ry, n_rx, K, H,
                                     W, C, p, vec, 16 / esize);
    cudaError_t e;
    if (dtype == kF32) {
        if ((e = cudaFuncSetAttribute(gather_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGatherSmem)) != cudaSuccess)
            return e;
        gather_kernel<float><<<tiles, kThreads, kGatherSmem, st>>>(P);
    } else {
        if ((e = cudaFuncSetAttribute(gather_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGatherSmem)) != cudaSuccess)
            return e;
        gather_kernel<uint8_t><<<tiles, kThreads, kGatherSmem, st>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_aggregate(const float* groups, const int32_t* idx, const float* weights,
                             int n_ry, int n_rx, int K, int H, int W, int C, int p, float* out,
                             float* wsum, cudaStream_t st) {
    cudaError_t e;
    const size_t out_bytes = (size_t)H * W * C * sizeof(float);
    const long long n_patch = (long long)n_ry * n_rx * K;
    // weights: histogram over top-left corners (in the output image, which
    // is cleared again afterwards), then a p x p box filter into wsum
    if ((e = cudaMemsetAsync(out, 0, out_bytes, st)) != cudaSuccess) return e;
    {
        const TileParams P = make_params(nullptr, nullptr, idx, weights, nullptr, nullptr, n_ry,
                                         n_rx, K, H, W, C, p, false, 1);
        long long blocks = (n_patch + kThreads - 1) / kThreads;
        if (blocks > 152LL * 8) blocks = 152LL * 8;
        if (blocks > 0) weight_hist_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(P, out);
        const dim3 grid((W + kBoxTile - 1) / kBoxTile, (H + kBoxTile - 1) / kBoxTile);
        weight_box_kernel<<<grid, kBoxTile * 8, 0, st>>>(out, wsum, H, W, p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(out, 0, out_bytes, st)) != cudaSuccess) return e;
    if (n_patch > 0) {
        // vectors: output pixel quads (W % 4 == 0, aligned buffers), one or four channels
        const bool vec = (C == 1 || C == 4) && W % 4 == 0 &&
                         reinterpret_cast<uintptr_t>(groups) % 16 == 0 &&
                         reinterpret_cast<uintptr_t>(out) % 16 == 0 &&
                         reinterpret_cast<uintptr_t>(wsum) % 16 == 0;
        const TileParams P = make_params(nullptr, const_cast<float*>(groups), idx, weights, out,
                                         wsum, n_ry, n_rx, K, H, W, C, p, vec, 4);
        long long blocks = (n_patch * 32 + kThreads - 1) / kThreads;
        if (blocks > 152LL * 8) blocks = 152LL * 8;
        aggregate_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(P);
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
    if ((long long)n_ry * n_rx == 0) return BM_OK;
    if (!img || !idx || !out_groups) return set_error(BM_ERR_INVALID, "null pointer");
    DevGuard dg(ctx_device(ctx));
    const cudaError_t e = launch_gather_groups(img, dtype == BM_U8 ? kU8 : kF32, idx, out_groups,
                                               n_ry, n_rx, K, H, W, C, patch,
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
