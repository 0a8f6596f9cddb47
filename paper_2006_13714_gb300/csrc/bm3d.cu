// bm3d.cu -- 3-D block matching across channels (§IV: 3-D Self-Convolution on
// patches of depth d < C channels, searched across channels, the channel sum
// S(.) omitted).
//
// A 3-D patch at (y, x, c) holds X[y + u][x + v][c + t], u, v < p, t < d.
// References: the spatial stride grid of block matching at every channel
// offset c_r in [0, C - d], reference index (ry * n_rx + rx) * (C - d + 1) + c_r.
// Candidates: the clipped spatial search window of block matching at every
// channel offset.  Output: the K nearest by (distance, offset), offset =
// (y * W + x) * C + c (the flat HWC index of the patch's first element).
// uint8 distances are exact (integers below 2^24); float32 distances are
// float32 sums of squared differences.
//
// Two kernels.  uint8 with a patch side of 4 or 8 runs bm3d_u8_kernel (the
// Self-Convolution identity in exact integers, dp4a on packed bytes; below).
// Every other shape runs bm3d_kernel on float32 squared differences.
//
// GB300 layout of the work (CUDA cores).  One block per tile_h x 8 tile of
// the spatial reference grid; tile_h is as small as keeps every warp busy, so
// the launch has many blocks and a short last wave.  The union of the tile's
// windows (all channels) is staged in shared memory channel-planar (plane stride 11 mod 32 words, row
// pitch equal to the window width mod 32), so the lanes of a warp, holding
// consecutive (column, channel offset) candidates, read distinct banks.  One
// warp per (reference, channel offset).  A lane evaluates R = 4 vertically
// adjacent candidates at once: per patch column and channel it loads the
// P + R - 1 candidate values of that column once and the P reference values
// (a broadcast), and forms R distances from them.  The reference therefore
// stays in shared memory, registers stay low enough for two blocks per SM,
// and the loads per candidate fall from p^2 d to (P + R - 1 + P) p d / R.
// The warp keeps its K best (distance, offset) keys one per lane in rank
// order; a ballot against the K-th screens 32 candidates, and each one that
// beats it is inserted at its rank (ballot count) with one shuffle of the
// list.
#include "bm.h"
#include "bm_internal.h"

#include <algorithm>
#include <climits>
#include <string>

namespace bm {
namespace {

constexpr int kTile3 = 8;
constexpr int kThreads3 = 384;
constexpr int kRows3 = 4;  // vertically adjacent candidates evaluated by one lane
constexpr int kMaxK3 = 32;
constexpr int kMaxElems3 = 128;
constexpr int kSmemLimit3 = 200 * 1024;  // two blocks per SM up to 113 KB
constexpr unsigned long long kEmpty3 = ~0ull;

struct Bm3dParams {
    const void* img;
    int32_t* out_idx;   // [n_ry*n_rx*nc][K]
    void* out_dist;     // int32 (uint8) / float32 (float32)
    int H, W, C, p, h, s, K, n_ry, n_rx, Hc, Wc, nc, tiles_x;
    int tile_h;         // reference rows per tile (the tile is tile_h x 8 references)
};

// Channel-plane stride for a plane of n words: n rounded up to 11 mod 32.
__host__ __device__ __forceinline__ int plane_stride(int n) { return n + ((11 - (n & 31)) & 31); }
// Region row pitch for n columns: n rounded up to the window width w mod 32.
__host__ __device__ __forceinline__ int row_pitch(int n, int w) { return n + ((w - n) & 31); }

template <int P, int D, bool kU8>
__global__ void __launch_bounds__(kThreads3, 2) bm3d_kernel(const Bm3dParams Q) {
    constexpr int R = kRows3, NW = P + R - 1;
    extern __shared__ __align__(16) float sreg[];
    const int ty = blockIdx.x / Q.tiles_x, tx = blockIdx.x - ty * Q.tiles_x;
    const int ry0 = ty * Q.tile_h, rx0 = tx * kTile3;
    const int ry1 = min(ry0 + Q.tile_h, Q.n_ry) - 1, rx1 = min(rx0 + kTile3, Q.n_rx) - 1;
    const int Y0 = max(0, ry0 * Q.s - Q.h), X0 = max(0, rx0 * Q.s - Q.h);
    const int Y1 = min(Q.Hc - 1, ry1 * Q.s + Q.h) + P, X1 = min(Q.Wc - 1, rx1 * Q.s + Q.h) + P;
    // R - 1 zero rows below the region: the last row group of a window reads
    // them for candidates past its end, whose results are dropped.
    const int C = Q.C, nrow = Y1 - Y0, srow = nrow + R - 1, gpitch = (X1 - X0) * C;
    const int ncol = row_pitch(X1 - X0, 2 * Q.h + 1);  // words between region rows
    const int ps = plane_stride(srow * ncol);          // words between channel planes
    for (int i = threadIdx.x; i < srow * gpitch; i += blockDim.x) {
        const int r = i / gpitch, e = i - r * gpitch;
        const int x = e / C, c = e - x * C;
        float v = 0.f;
        if (r < nrow) {
            const size_t g = ((size_t)(Y0 + r) * Q.W + X0) * C + e;
            v = kU8 ? (float)static_cast<const uint8_t*>(Q.img)[g] : static_cast<const float*>(Q.img)[g];
        }
        sreg[c * ps + r * ncol + x] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ntx = rx1 - rx0 + 1, nref = (ry1 - ry0 + 1) * ntx * Q.nc;
    const int K = Q.K;
    for (int rl = warp; rl < nref; rl += nwarps) {
        const int rs = rl / Q.nc, cr = rl - rs * Q.nc;
        const int ry = ry0 + rs / ntx, rx = rx0 + rs % ntx;
        const int yr = ry * Q.s, xr = rx * Q.s;
        const float* rb = sreg + cr * ps + (yr - Y0) * ncol + (xr - X0);
        const int cy0 = max(0, yr - Q.h), cy1 = min(Q.Hc - 1, yr + Q.h);
        const int cx0 = max(0, xr - Q.h), cx1 = min(Q.Wc - 1, xr + Q.h);
        const int wxc = (cx1 - cx0 + 1) * Q.nc;
        const int nitem = ((cy1 - cy0 + R) / R) * wxc;  // (row group, column, channel offset)
        unsigned long long mine = kEmpty3, kth = kEmpty3;
        for (int j0 = 0; j0 < nitem; j0 += 32) {
            const int j = j0 + lane;
            const bool live = j < nitem;
            float acc[R];
#pragma unroll
            for (int i = 0; i < R; ++i) acc[i] = 0.f;
            int yc = cy0, xc = cx0, cc = 0;
            if (live) {
                const int jb = j / wxc, rem = j - jb * wxc;
                const int jx = rem / Q.nc;
                cc = rem - jx * Q.nc;
                yc = cy0 + jb * R;
                xc = cx0 + jx;
                const float* cb = sreg + cc * ps + (yc - Y0) * ncol + (xc - X0);
#pragma unroll
                for (int t = 0; t < D; ++t)
#pragma unroll
                    for (int v = 0; v < P; ++v) {
                        float w[NW], rr[P];
#pragma unroll
                        for (int u = 0; u < NW; ++u) w[u] = cb[t * ps + u * ncol + v];
#pragma unroll
                        for (int u = 0; u < P; ++u) rr[u] = rb[t * ps + u * ncol + v];
#pragma unroll
                        for (int u = 0; u < P; ++u)
#pragma unroll
                            for (int i = 0; i < R; ++i) {
                                const float df = rr[u] - w[u + i];
                                acc[i] = fmaf(df, df, acc[i]);
                            }
                    }
            }
#pragma unroll
            for (int i = 0; i < R; ++i) {
                unsigned long long key = kEmpty3;
                if (live && yc + i <= cy1) {
                    const unsigned off = (unsigned)(((yc + i) * Q.W + xc) * C + cc);
                    key = kU8 ? ((unsigned long long)(unsigned)acc[i] << 32) | off
                              : ((unsigned long long)__float_as_uint(acc[i]) << 32) | off;
                }
                warp_list_offer(key, mine, kth, lane, K);
            }
        }
        if (lane < K) {
            const size_t ref_id = ((size_t)ry * Q.n_rx + rx) * Q.nc + cr;
            Q.out_idx[ref_id * K + lane] = mine == kEmpty3 ? -1 : (int32_t)(unsigned)mine;
            if (kU8)
                static_cast<int32_t*>(Q.out_dist)[ref_id * K + lane] =
                    mine == kEmpty3 ? INT_MAX : (int32_t)(unsigned)(mine >> 32);
            else
                static_cast<float*>(Q.out_dist)[ref_id * K + lane] =
                    mine == kEmpty3 ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(mine >> 32));
        }
    }
}

// ---------------------------------------------------------------------------
// uint8, patch side a multiple of 4: the distance through the Self-Convolution
// identity in exact integers (Lemma 2 applied to the 3-D patches),
//   d(r, j) = ||X_r||^2 + ||X_j||^2 - 2 <X_r, X_j>,
// four pixels at a time with dp4a on bytes.  The region is staged as bytes,
// channel-planar (plane stride 8 mod 32 words, one spare word per row for the
// shifted reads).  A patch row of a candidate at any column is two funnel
// shifts of three loaded words; the reference patch sits in registers as
// p^2 d / 4 words.  A lane evaluates R = 8 vertically adjacent candidates: each
// window row it loads feeds the cross terms of up to R candidates and one
// row norm, and the candidates' norms are sliding sums of those row norms.
// Every partial sum is an integer below 2^24, so the result equals the
// floating-point path's bit for bit.
constexpr int kRowsI = 8;
constexpr int kThreadsI = 256;

// Channel-plane stride (words) for the byte region: n rounded up to 8 mod 32.
__host__ __device__ __forceinline__ int plane_stride_u8(int n) { return n + ((8 - (n & 31)) & 31); }
// Words per byte-region row of n columns: the columns plus one spare word.
__host__ __device__ __forceinline__ int row_words_u8(int n) { return (n + 3) / 4 + 1; }

template <int P, int D>
__global__ void __launch_bounds__(kThreadsI, 2) bm3d_u8_kernel(const Bm3dParams Q) {
    static_assert(P % 4 == 0, "patch side must be a multiple of 4");
    constexpr int R = kRowsI, NW = P + R - 1, NQ = P / 4;
    extern __shared__ __align__(16) uint32_t sw[];
    const int ty = blockIdx.x / Q.tiles_x, tx = blockIdx.x - ty * Q.tiles_x;
    const int ry0 = ty * Q.tile_h, rx0 = tx * kTile3;
    const int ry1 = min(ry0 + Q.tile_h, Q.n_ry) - 1, rx1 = min(rx0 + kTile3, Q.n_rx) - 1;
    const int Y0 = max(0, ry0 * Q.s - Q.h), X0 = max(0, rx0 * Q.s - Q.h);
    const int Y1 = min(Q.Hc - 1, ry1 * Q.s + Q.h) + P, X1 = min(Q.Wc - 1, rx1 * Q.s + Q.h) + P;
    const int C = Q.C, nrow = Y1 - Y0, ncol = X1 - X0, gpitch = ncol * C;
    const int pw = row_words_u8(ncol);                 // words between region rows
    const int ps = plane_stride_u8((nrow + R - 1) * pw);  // words between channel planes
    // zero the planes (the R - 1 rows below the region and the spare words
    // are read for candidates whose results are dropped), then stage
    for (int i = threadIdx.x; i < C * ps; i += blockDim.x) sw[i] = 0u;
    __syncthreads();
    unsigned char* sb = reinterpret_cast<unsigned char*>(sw);
    const uint8_t* im = static_cast<const uint8_t*>(Q.img);
    for (int i = threadIdx.x; i < nrow * gpitch; i += blockDim.x) {
        const int r = i / gpitch, e = i - r * gpitch;
        const int x = e / C, c = e - x * C;
        sb[4 * (c * ps + r * pw) + x] = im[((size_t)(Y0 + r) * Q.W + X0) * C + e];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ntx = rx1 - rx0 + 1, nref = (ry1 - ry0 + 1) * ntx * Q.nc;
    const int K = Q.K;
    for (int rl = warp; rl < nref; rl += nwarps) {
        const int rs = rl / Q.nc, cr = rl - rs * Q.nc;
        const int ry = ry0 + rs / ntx, rx = rx0 + rs % ntx;
        const int yr = ry * Q.s, xr = rx * Q.s;
        // reference patch rows as words (byte k of word q = column 4q + k)
        uint32_t ref[D][P][NQ];
        unsigned nr = 0u;
        {
            const int sh = 8 * ((xr - X0) & 3);
#pragma unroll
            for (int t = 0; t < D; ++t)
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    const uint32_t* rp = sw + (cr + t) * ps + (yr - Y0 + u) * pw + ((xr - X0) >> 2);
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        ref[t][u][q] = __funnelshift_r(rp[q], rp[q + 1], sh);
                        nr = __dp4a(ref[t][u][q], ref[t][u][q], nr);
                    }
                }
        }
        const int cy0 = max(0, yr - Q.h), cy1 = min(Q.Hc - 1, yr + Q.h);
        const int cx0 = max(0, xr - Q.h), cx1 = min(Q.Wc - 1, xr + Q.h);
        const int wxc = (cx1 - cx0 + 1) * Q.nc;
        const int nitem = ((cy1 - cy0 + R) / R) * wxc;  // (row group, column, channel offset)
        unsigned long long mine = kEmpty3, kth = kEmpty3;
        for (int j0 = 0; j0 < nitem; j0 += 32) {
            const int j = j0 + lane;
            const bool live = j < nitem;
            unsigned cross[R], sq[NW];
#pragma unroll
            for (int i = 0; i < R; ++i) cross[i] = 0u;
#pragma unroll
            for (int u = 0; u < NW; ++u) sq[u] = 0u;
            int yc = cy0, xc = cx0, cc = 0;
            if (live) {
                const int jb = j / wxc, rem = j - jb * wxc;
                const int jx = rem / Q.nc;
                cc = rem - jx * Q.nc;
                yc = cy0 + jb * R;
                xc = cx0 + jx;
                const int sh = 8 * ((xc - X0) & 3);
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const uint32_t* cp = sw + (cc + t) * ps + (yc - Y0) * pw + ((xc - X0) >> 2);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        uint32_t raw[NQ + 1], cw[NQ];
#pragma unroll
                        for (int q = 0; q <= NQ; ++q) raw[q] = cp[w * pw + q];
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            cw[q] = __funnelshift_r(raw[q], raw[q + 1], sh);
                            sq[w] = __dp4a(cw[q], cw[q], sq[w]);
                        }
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            const int u = w - i;  // patch row of window row w for candidate i
                            if (u >= 0 && u < P) {
#pragma unroll
                                for (int q = 0; q < NQ; ++q) cross[i] = __dp4a(ref[t][u][q], cw[q], cross[i]);
                            }
                        }
                    }
                }
            }
            // candidate norms: sliding sums of P row norms
            unsigned nj = 0u;
#pragma unroll
            for (int u = 0; u < P; ++u) nj += sq[u];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (i > 0) nj += sq[i + P - 1] - sq[i - 1];
                unsigned long long key = kEmpty3;
                if (live && yc + i <= cy1) {
                    const unsigned d = nr + nj - 2u * cross[i];
                    const unsigned off = (unsigned)(((yc + i) * Q.W + xc) * C + cc);
                    key = ((unsigned long long)d << 32) | off;
                }
                warp_list_offer(key, mine, kth, lane, K);
            }
        }
        if (lane < K) {
            const size_t ref_id = ((size_t)ry * Q.n_rx + rx) * Q.nc + cr;
            Q.out_idx[ref_id * K + lane] = mine == kEmpty3 ? -1 : (int32_t)(unsigned)mine;
            static_cast<int32_t*>(Q.out_dist)[ref_id * K + lane] =
                mine == kEmpty3 ? INT_MAX : (int32_t)(unsigned)(mine >> 32);
        }
    }
}

using Bm3dKernel = void (*)(Bm3dParams);

// uint8 shapes served by the integer kernel (patch side 4 or 8).
Bm3dKernel pick3_u8(int p, int d) {
#define BM3_CASE(PP, DD) \
    if (p == PP && d == DD) return bm3d_u8_kernel<PP, DD>;
    BM3_CASE(4, 1) BM3_CASE(4, 2) BM3_CASE(4, 3) BM3_CASE(4, 4) BM3_CASE(8, 1) BM3_CASE(8, 2)
#undef BM3_CASE
    return nullptr;
}

Bm3dKernel pick3(int p, int d, bool u8) {
#define BM3_CASE(PP, DD) \
    if (p == PP && d == DD) return u8 ? bm3d_kernel<PP, DD, true> : bm3d_kernel<PP, DD, false>;
    BM3_CASE(1, 1) BM3_CASE(2, 1) BM3_CASE(3, 1) BM3_CASE(4, 1) BM3_CASE(5, 1) BM3_CASE(6, 1)
    BM3_CASE(7, 1) BM3_CASE(8, 1)
    BM3_CASE(1, 2) BM3_CASE(2, 2) BM3_CASE(3, 2) BM3_CASE(4, 2) BM3_CASE(5, 2)
    BM3_CASE(1, 3) BM3_CASE(2, 3) BM3_CASE(3, 3) BM3_CASE(4, 3)
    BM3_CASE(2, 4) BM3_CASE(3, 4) BM3_CASE(4, 4)
    BM3_CASE(6, 2) BM3_CASE(7, 2) BM3_CASE(8, 2) BM3_CASE(5, 3) BM3_CASE(6, 3) BM3_CASE(5, 4)
#undef BM3_CASE
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

int bm_match_3d(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                int depth, int window, int stride, int K, int32_t* out_idx, void* out_dist,
                bm_stream stream) {
    if (!ctx) return set_error(BM_ERR_INVALID, "null context");
    if (dtype != BM_U8 && dtype != BM_F32) return set_error(BM_ERR_INVALID, "unknown dtype");
    if (H < 1 || W < 1 || C < 1 || C > kMaxC || patch < 1 || patch > H || patch > W ||
        depth < 1 || depth > C || window < 1 || window % 2 == 0 || window > kMaxWindow ||
        stride < 1 || K < 1 || K > kMaxK)
        return set_error(BM_ERR_INVALID, "invalid geometry, depth or K");
    if (!img || !out_idx || !out_dist) return set_error(BM_ERR_INVALID, "null pointer");
    if ((long long)H * W * C >= (1LL << 31))
        return set_error(BM_ERR_UNSUPPORTED, "H*W*C must be below 2^31");
    if (patch * patch * depth > kMaxElems3 || K > kMaxK3)
        return set_error(BM_ERR_UNSUPPORTED, "3-D matching serves patch*patch*depth <= 128 and K <= 32");
    const bool u8 = dtype == BM_U8;
    const Bm3dKernel kint = u8 ? pick3_u8(patch, depth) : nullptr;
    const Bm3dKernel kern = kint ? kint : pick3(patch, depth, u8);
    if (!kern) return set_error(BM_ERR_UNSUPPORTED, "patch / depth shape not instantiated");
    const int threads = kint ? kThreadsI : kThreads3;
    Bm3dParams Q{};
    Q.img = img; Q.out_idx = out_idx; Q.out_dist = out_dist;
    Q.H = H; Q.W = W; Q.C = C; Q.p = patch; Q.h = (window - 1) / 2; Q.s = stride; Q.K = K;
    Q.n_ry = (H - patch) / stride + 1; Q.n_rx = (W - patch) / stride + 1;
    Q.Hc = H - patch + 1; Q.Wc = W - patch + 1; Q.nc = C - depth + 1;
    // Tiles of tile_h x 8 references: the fewest rows that still give every
    // warp two (reference, channel offset) tasks.  Short tiles make many
    // blocks, so the last wave of blocks is a small part of the launch.
    Q.tile_h = std::min(kTile3, (2 * (threads / 32) + kTile3 * Q.nc - 1) / (kTile3 * Q.nc));
    Q.tiles_x = (Q.n_rx + kTile3 - 1) / kTile3;
    const int tiles = ((Q.n_ry + Q.tile_h - 1) / Q.tile_h) * Q.tiles_x;
    const int rows = std::min(H, (Q.tile_h - 1) * stride + 2 * Q.h + patch);
    const int cols = std::min(W, (kTile3 - 1) * stride + 2 * Q.h + patch);
    const size_t smem =
        kint ? (size_t)plane_stride_u8((rows + kRowsI - 1) * row_words_u8(cols)) * C * sizeof(uint32_t)
             : (size_t)plane_stride((rows + kRows3 - 1) * row_pitch(cols, 2 * Q.h + 1)) * C * sizeof(float);
    if (smem > (size_t)kSmemLimit3)
        return set_error(BM_ERR_UNSUPPORTED, "search region does not fit in shared memory");
    DevGuard dg(ctx_device(ctx));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        kern<<<tiles, threads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(Q);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("3-D match launch: ") + cudaGetErrorString(e)).c_str());
    return BM_OK;
}

}  // extern "C"
