// bm_static.cu -- bm_match_static: block matching that allocates nothing.
//
// This entry point serves callers that must not allocate device memory while
// they run: cudaMalloc / cudaFree synchronise the whole device (a stall in a
// latency-bound loop), and in a process whose device memory is already held
// by another allocator a fresh allocation can fail part-way through a run.
// Every intermediate buffer of the tensor-core path comes from one fixed
// array in device memory.  The array belongs to this file's module: CUDA
// loads modules lazily by default, so the array is reserved by the first
// symbol lookup on a device (bm_static_init, or the first bm_match_static
// there), or at start-up under CUDA_MODULE_LOADING=EAGER.  The kernels are
// the ones bm_match runs, on the same geometry, so the results are the same.
//
// Timeouts: a bounded device wait of the tensor-core kernel that runs out
// leaves the job's outputs incomplete.  The kernel then records its code in
// a sticky per-device fault word (outside the part each call clears), which
// bm_static_check reads and clears.
//
// Limits and sharing: the array holds BM_STATIC_SCRATCH_BYTES; larger jobs
// are rejected with BM_ERR_TOO_LARGE before anything is launched.  All calls
// on a device share the array, so calls that overlap on the GPU race.
#include "bm.h"
#include "bm_internal.h"

#include <cstdio>
#include <atomic>
#include <mutex>
#include <string>

namespace bm {
namespace {

// The scratch array.  One copy per device, reserved at module load.
static __device__ __align__(256) unsigned char g_scratch[BM_STATIC_SCRATCH_BYTES];
// Sticky timeout word: the first timeout code since the last bm_static_check.
static __device__ int g_fault;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_base[kMaxDevices] = {};
int* g_fault_ptr[kMaxDevices] = {};
std::atomic<int> g_inject{0};  // test hook: the next call's kernel withholds its first stage

size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte layout inside the array.  The 256-byte header at offset 0 holds the
// tensor-core status word (int, offset 0), the centring offset (float,
// offset 16) and the re-rank counters (4 x u64, offset 32); the header is the
// only part that must start at zero, and each call clears it.
struct Layout {
    size_t plane0, plane1, nrm, nsp, pool_idx, pool_score, split, total;
    int parts;  // column parts of the class (their part lists follow the pool)
};
constexpr size_t kHeader = 256;
constexpr size_t kCenterOff = 16;
constexpr size_t kCountersOff = 32;

Layout layout(const Geom& g) {
    Layout l{};
    size_t off = kHeader;
    if (tc_supported(g)) {
        l.plane0 = off; off += round256(plane_bytes(g));
        l.plane1 = off; off += g.dtype == kF32 ? round256(plane_bytes(g)) : 0;
        l.nrm = off; off += round256(nrm_bytes(g));
        l.nsp = off; off += round256(nsp_bytes(g));
        l.pool_idx = off; off += g.dtype == kF32 ? round256((size_t)g.nR * g.L * 4) : 0;
        l.pool_score = off; off += g.dtype == kF32 ? round256((size_t)g.nR * g.L * 4) : 0;
        l.parts = tc_column_parts(g);
        const size_t nlist = (size_t)g.nR * (g.dtype == kF32 ? g.L : g.K);
        l.split = off; off += l.parts > 1 ? 2 * round256((size_t)l.parts * nlist * 4) : 0;
    }
    l.total = off;
    return l;
}

int check_args(Geom& g, int H, int W, int C, int dtype, int p, int win, int s, int K) {
    int rc = make_geom(g, H, W, C, dtype, p, win, s, K);
    if (rc == BM_ERR_INVALID) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "invalid arguments: H=%d W=%d C=%d dtype=%d patch=%d window=%d stride=%d K=%d "
                 "(need 1<=patch<=min(H,W), odd window<=%d, stride>=1, 1<=K<=%d, 1<=C<=%d)",
                 H, W, C, dtype, p, win, s, K, kMaxWindow, kMaxK, kMaxC);
        return set_error(rc, buf);
    }
    if (rc == BM_ERR_UNSUPPORTED)
        return set_error(rc, "unsupported: patch*patch*C must be <= 256 and H*W < 2^31");
    return rc;
}

// Device addresses of the array and of the fault word on the current
// device; the first call per device looks them up (which loads the module).
int scratch_base(void** out, int** fault) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_error(BM_ERR_CUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    if (dev < 0 || dev >= kMaxDevices) return set_error(BM_ERR_UNSUPPORTED, "device index >= 64");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void* ptr = nullptr;
        void* fptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&fptr, g_fault);
        if (e != cudaSuccess || !ptr || !fptr)
            return set_error(BM_ERR_CUDA,
                             (std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)).c_str());
        g_base[dev] = ptr;
        g_fault_ptr[dev] = static_cast<int*>(fptr);
    }
    *out = g_base[dev];
    if (fault) *fault = g_fault_ptr[dev];
    return BM_OK;
}

int launch_fail(cudaError_t e, const char* where) {
    return set_error(BM_ERR_CUDA, (std::string(where) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" size_t bm_static_scratch_bytes(int H, int W, int C, bm_dtype dtype, int patch,
                                          int window, int stride, int K) {
    Geom g;
    if (make_geom(g, H, W, C, (int)dtype, patch, window, stride, K) != 0) return 0;
    return layout(g).total;
}

extern "C" int bm_match_static(const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                               int window, int stride, int K, int32_t* out_idx, void* out_dist,
                               bm_stream stream) {
    Geom g;
    int rc = check_args(g, H, W, C, (int)dtype, patch, window, stride, K);
    if (rc != BM_OK) return rc;
    if (!img || !out_idx || !out_dist) return set_error(BM_ERR_INVALID, "null pointer argument");
    const Layout l = layout(g);
    if (l.total > BM_STATIC_SCRATCH_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "job too large for bm_match_static: needs %zu bytes of scratch, the static "
                 "array holds %zu",
                 l.total, (size_t)BM_STATIC_SCRATCH_BYTES);
        return set_error(BM_ERR_TOO_LARGE, buf);
    }
    void* base = nullptr;
    int* fault = nullptr;
    if ((rc = scratch_base(&base, &fault)) != BM_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* b = static_cast<char*>(base);
    cudaError_t e;
    if ((e = cudaMemsetAsync(b, 0, kHeader, st)) != cudaSuccess) return launch_fail(e, "scratch reset");
    if (!tc_supported(g)) {
        // Geometries outside the tensor-core kernel's tiling: the direct
        // kernel, which needs no scratch (as bm_match does).
        if ((e = launch_direct(g, img, out_idx, out_dist, st)) != cudaSuccess)
            return launch_fail(e, "direct kernel launch");
        return BM_OK;
    }
    uint16_t* p0 = reinterpret_cast<uint16_t*>(b + l.plane0);
    uint16_t* p1 = g.dtype == kF32 ? reinterpret_cast<uint16_t*>(b + l.plane1) : nullptr;
    void* nrm = b + l.nrm;
    uint16_t* nsp = reinterpret_cast<uint16_t*>(b + l.nsp);
    float* center = reinterpret_cast<float*>(b + kCenterOff);
    auto* counters = reinterpret_cast<unsigned long long*>(b + kCountersOff);
    if ((e = launch_center(g, img, center, st)) != cudaSuccess) return launch_fail(e, "centre kernel launch");
    if ((e = launch_planes(g, img, center, p0, p1, st)) != cudaSuccess)
        return launch_fail(e, "plane kernel launch");
    if ((e = launch_boxfilter(g, img, center, nrm, nsp, st)) != cudaSuccess)
        return launch_fail(e, "box filter launch");
    TcArgs a{};
    a.plane0 = p0;
    a.plane1 = p1;
    a.nrm = nrm;
    a.nsp = nsp;
    a.status = reinterpret_cast<int*>(b);
    a.fault = fault;
    a.inject = g_inject.exchange(0);
    if (g.dtype == kU8) {
        a.out_idx = out_idx;
        a.out_dist = static_cast<int32_t*>(out_dist);
    } else {
        a.pool_idx = reinterpret_cast<int32_t*>(b + l.pool_idx);
        a.pool_score = reinterpret_cast<float*>(b + l.pool_score);
    }
    if (l.parts > 1) {  // column parts: the parts' lists, merged by the launch
        const size_t nlist = (size_t)g.nR * (g.dtype == kF32 ? g.L : g.K);
        a.wsplit = l.parts;
        a.split_idx = reinterpret_cast<int32_t*>(b + l.split);
        a.split_val = reinterpret_cast<int32_t*>(b + l.split + round256((size_t)l.parts * nlist * 4));
    }
    if ((e = launch_tc(g, a, st)) != cudaSuccess) return launch_fail(e, "tensor-core kernel launch");
    if (g.dtype == kF32) {
        e = launch_rerank(g, static_cast<const float*>(img), static_cast<const float*>(nrm),
                          a.pool_idx, a.pool_score, out_idx, static_cast<float*>(out_dist),
                          counters, st);
        if (e != cudaSuccess) return launch_fail(e, "re-rank kernel launch");
    }
    return BM_OK;
}

extern "C" int bm_static_init(void) {
    void* base = nullptr;
    return scratch_base(&base, nullptr);
}

extern "C" int bm_static_check(bm_stream stream) {
    void* base = nullptr;
    int* fault = nullptr;
    int rc = scratch_base(&base, &fault);
    if (rc != BM_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int v = 0;  // a host int: nothing is allocated
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, fault, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return launch_fail(e, "reading the static fault word");
    if (v == 0) return BM_OK;
    if ((e = cudaMemsetAsync(fault, 0, sizeof(int), st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return launch_fail(e, "clearing the static fault word");
    return set_error(BM_ERR_TIMEOUT, timeout_message(v));
}

extern "C" int bm_static_set_fault_injection(int mode) {
    if (mode != 0 && mode != 1) return set_error(BM_ERR_INVALID, "unknown fault injection mode");
    g_inject.store(mode);
    return BM_OK;
}
