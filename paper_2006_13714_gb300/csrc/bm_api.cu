// bm_api.cu -- host runtime and C ABI of the block-matching library.
//
// Context = one device, a device-memory budget for the library's own
// workspace, a per-stream workspace cache, device counters, and a serving
// loop (host thread) that admits submitted requests under the budget and
// runs them concurrently on a small set of streams.
#include "bm_internal.h"
#include "../../include/bm.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <fstream>
#include <map>
#include <sstream>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace bm {

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Float32 pool L: the candidates per reference the tensor-core pass keeps for
// the re-rank.  A reference whose whole pool lies inside the re-rank's error
// band is recomputed over its window (every candidate's direct distance), so
// the pool needs room beyond K for the candidates whose estimates fall
// within the error of the K-th.  L = K + 8 (rounded up to 8) by default; a
// larger pool costs selection work in the tensor-core pass (a looser
// threshold, more appends) and pays where that recompute is frequent:
// - four or eight channels: K + 16 up to K 40, K + 24 above;
// - one to three channels at windows of 45 or more: K + 16 for K <= 24
//   (32 entries: the register lists' full width) and for K > 40.
// Measured recompute rates at L = K + 8 (1024^2 images): four-channel K 70
// 8-15 %, window 61 K 16 5 %, one-channel window 61 K 70 8 %; at K + 16/24
// under 0.3 %.  Times (1024^2, float32, matching plus re-rank): four-channel
// p 8 window 61 K 70 15.3 -> 9.9 ms, K 16 6.1 -> 3.8 ms; one-channel window
// 61 K 16 1.65 -> 1.16 ms.  On the 512^2 window-39 K 16 batch the larger pool
// cost 9 % (recomputes were 0.35 %), so it stays at K + 8 there.
static int pool_extra(int K, int C, int h) {
    if (C >= 4) return K <= 40 ? 16 : 24;
    if (2 * h + 1 >= 45 && (K <= 24 || K > 40)) return 16;
    return 8;
}

// The larger pool is taken only when its tensor-core geometry is no worse in
// any of these: no more column parts, no fewer tile slots or candidate
// columns per MMA, no smaller append buffer (16 entries merge after every
// block), A not moved to tensor memory, the same tile shape.
static bool no_worse(const TcShape& b, const TcShape& a) {
    return b.xs <= a.xs && b.ns >= a.ns && b.kcols >= a.kcols && b.kbuf >= a.kbuf && b.ts <= a.ts &&
           b.ty == a.ty && b.tx == a.tx;
}

int make_geom(Geom& g, int H, int W, int C, int dtype, int p, int win, int s, int K) {
    if (H < 1 || W < 1 || C < 1 || C > kMaxC || p < 1 || p > H || p > W) return BM_ERR_INVALID;
    if (win < 1 || (win % 2) == 0 || win > kMaxWindow || s < 1 || K < 1 || K > kMaxK)
        return BM_ERR_INVALID;
    if (dtype != kU8 && dtype != kF32) return BM_ERR_INVALID;
    if ((long long)H * W >= (1ll << 31)) return BM_ERR_UNSUPPORTED;
    if (p * p * C > kMaxPatchElems) return BM_ERR_UNSUPPORTED;
    g.H = H; g.W = W; g.C = C; g.dtype = dtype;
    g.p = p; g.win = win; g.h = (win - 1) / 2; g.s = s; g.K = K;
    g.n_ry = (H - p) / s + 1;
    g.n_rx = (W - p) / s + 1;
    g.nR = g.n_ry * g.n_rx;
    g.Hc = H - p + 1;
    g.Wc = W - p + 1;
    g.Cp = C == 1 ? 1 : C == 2 ? 2 : C <= 4 ? 4 : 8;
    int elems = p * g.Cp;
    g.pw = (elems + 7) / 8;
    if (g.pw > 1 && (g.pw & 1)) g.pw += 1;
    g.p_eff = g.pw == 1 ? round_up(p, 2) : p;
    // plane rows: room for the widest staged strip beyond the right edge
    g.plane_pitch = round_up(W * g.Cp + 8 * g.pw + 16, 8);
    g.plane_rows = H + g.p_eff + 8;
    g.L = dtype == kF32 ? std::min(160, round_up(K + 8, 8)) : 0;
    if (dtype == kF32) {
        // a larger pool where references often fall to a window recompute
        const int extra = pool_extra(K, C, g.h);
        if (extra > 8) {
            Geom big = g;
            big.L = std::min(160, round_up(K + extra, 8));
            TcShape a{}, b{};
            if (big.L > g.L && tc_shape(g, a) && tc_shape(big, b) && no_worse(b, a)) g.L = big.L;
        }
    }
    return BM_OK;
}

size_t plane_bytes(const Geom& g) { return (size_t)g.plane_rows * g.plane_pitch * 2; }
size_t nrm_bytes(const Geom& g) { return (size_t)g.Hc * g.Wc * 4; }
size_t pool_bytes(const Geom& g) { return g.dtype == kF32 ? (size_t)g.nR * g.L * 8 : 0; }
size_t nsp_bytes(const Geom& g) { return (size_t)g.Hc * g.Wc * 16; }

bool tc_supported(const Geom& g);  // selfconv_tc.cu

}  // namespace bm

using namespace bm;

namespace {

thread_local std::string t_last_error;

}  // namespace

namespace bm {
// Sets the calling thread's bm_last_error message; for entry points defined
// in other files of the library.
int set_error(int code, const char* msg) {
    t_last_error = msg;
    return code;
}

const char* timeout_message(int code) {
    static const char* const msgs[] = {
        "a bounded device wait of the tensor-core kernel ran out (unknown site)",
        "a bounded device wait of the tensor-core kernel ran out (stage free)",
        "a bounded device wait of the tensor-core kernel ran out (accumulator free)",
        "a bounded device wait of the tensor-core kernel ran out (stage filled)",
        "a bounded device wait of the tensor-core kernel ran out (accumulator filled)",
        "a bounded device wait of the tensor-core kernel ran out (A operand free)",
        "a bounded device wait of the tensor-core kernel ran out (tile staged)",
        "a bounded device wait of the tensor-core kernel ran out (A operand formed)"};
    const int site = code - 0x100;
    return msgs[site >= 1 && site <= 7 ? site : 0];
}
}  // namespace bm

namespace {

struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct GraphEntry {
    std::vector<bm_request> reqs;  // the job list the graph was captured for
    void* ws = nullptr;
    int algo = 0;
    size_t tc_jobs = 0;
    cudaGraphExec_t exec = nullptr;
};

struct Batch {
    cudaEvent_t ev;
    int slot;
    int ring;  // status ring entry: per-job error words (device) and their host copy
    size_t bytes;
    std::vector<uint64_t> ids;
};

struct Ticket {
    bm_request req;
    int status = BM_OK;
    std::string msg;  // bm_last_error text of a failed request (set at retire)
    bool admitted = false;
    bool done = false;
    size_t ws_bytes = 0;
    int slot = -1;
    void* ws = nullptr;
    cudaEvent_t ev = nullptr;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte layout of one tensor-core job's workspace.
struct WsLayout {
    size_t plane0, plane1, nrm, nsp, pool_idx, pool_score, status, split, total;
    int wsplit;
};

WsLayout ws_layout(const Geom& g) {
    WsLayout l{};
    size_t off = 0;
    l.plane0 = off; off += align256(plane_bytes(g));
    l.plane1 = off; off += g.dtype == kF32 ? align256(plane_bytes(g)) : 0;
    l.nrm = off; off += align256(nrm_bytes(g));
    l.nsp = off; off += align256(nsp_bytes(g));
    l.pool_idx = off; off += g.dtype == kF32 ? align256((size_t)g.nR * g.L * 4) : 0;
    l.pool_score = off; off += g.dtype == kF32 ? align256((size_t)g.nR * g.L * 4) : 0;
    l.status = off; off += 256;
    // window split: the parts' lists (offsets, then distances / score bits)
    l.wsplit = tc_window_split(g);
    const size_t nlist = (size_t)g.nR * (g.dtype == kF32 ? g.L : g.K);
    l.split = off; off += l.wsplit > 1 ? 2 * align256((size_t)l.wsplit * nlist * 4) : 0;
    l.total = off;
    return l;
}

}  // namespace

struct bm_ctx {
    int device = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    std::string tune_cache;                   // autotuner table file ("" = no tuning)
    std::mutex tune_mu;
    std::map<std::string, int> tune_table;    // class key -> tile configuration
    bm_algo algo = BM_ALGO_AUTO;
    std::mutex ws_mu;
    std::unordered_map<cudaStream_t, Workspace> ws;  // per-stream cache
    std::mutex graph_mu;
    std::unordered_map<cudaStream_t, GraphEntry> graphs;  // captured batches, per stream
    int* d_fault = nullptr;                          // sticky timeout word of the tensor-core kernel
    std::atomic<int> inject{0};                      // one-shot fault injection (test hook)
    unsigned long long* d_counters = nullptr;        // [0] overflow, [1] fp64 rechecks
    std::atomic<unsigned long long> matches{0}, refs{0}, tc_jobs{0};
    // stage timing
    std::atomic<int> timing{0};
    std::mutex tm_mu;
    struct EvPair { int stage; int n; cudaEvent_t a, b; };
    std::vector<EvPair> tm_pending;
    bm_timing tm_total{};
    // host-buffer path
    std::mutex host_mu;
    cudaStream_t host_stream = nullptr;
    void* h_dev_img = nullptr; size_t h_dev_img_bytes = 0;
    // bm_match_host_batch: two pipelines (stream + device staging each)
    cudaStream_t hb_stream[2] = {nullptr, nullptr};
    void* hb_buf[2] = {nullptr, nullptr};
    size_t hb_bytes[2] = {0, 0};
    void* h_dev_out = nullptr; size_t h_dev_out_bytes = 0;
    // serving
    static constexpr int kSlots = 4;
    static constexpr int kMaxBatch = 64;  // requests per admitted batch
    static constexpr int kRing = 2 * kSlots;  // batches in flight at most
    cudaStream_t slot_stream[kSlots] = {};
    int slot_busy[kSlots] = {};
    // per-job error words of the batches in flight: entry r holds kMaxBatch
    // words on the device and their pinned host copy (read at retire)
    int* d_ring = nullptr;
    int* h_ring = nullptr;
    bool ring_busy[kRing] = {};
    cudaStream_t aux_stream = nullptr;  // reads of the fault word and counters
    std::mutex br_mu;
    std::unordered_map<cudaStream_t, std::vector<cudaStream_t>> branches;  // class branches per stream
    std::mutex q_mu;
    std::condition_variable q_cv;
    std::deque<uint64_t> pending;
    std::vector<Batch> batches;  // admitted, not yet retired
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
};

namespace {

int fail(int code, const std::string& msg) {
    t_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(BM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int validate(const bm_request& r, Geom& g) {
    int rc = make_geom(g, r.H, r.W, r.C, (int)r.dtype, r.patch, r.window, r.stride, r.K);
    if (rc == BM_ERR_INVALID) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "invalid arguments: H=%d W=%d C=%d dtype=%d patch=%d window=%d stride=%d K=%d "
                 "(need 1<=patch<=min(H,W), odd window<=%d, stride>=1, 1<=K<=%d, 1<=C<=%d)",
                 r.H, r.W, r.C, (int)r.dtype, r.patch, r.window, r.stride, r.K, kMaxWindow,
                 kMaxK, kMaxC);
        return fail(rc, buf);
    }
    if (rc == BM_ERR_UNSUPPORTED)
        return fail(rc, "unsupported: patch*patch*C must be <= 256 and H*W < 2^31");
    if (!r.img || !r.out_idx || !r.out_dist) return fail(BM_ERR_INVALID, "null pointer argument");
    return BM_OK;
}

bool use_tc(bm_ctx* ctx, const Geom& g) {
    if (ctx->algo == BM_ALGO_DIRECT) return false;
    return tc_supported(g);
}

size_t job_ws_bytes(bm_ctx* ctx, const Geom& g) {
    return use_tc(ctx, g) ? ws_layout(g).total : 0;
}

// Run `launch` on st; with stage timing on, bracket it with two events.
// nlaunch (optional) = kernel launches the bracket holds, read after launch().
template <class F>
cudaError_t timed(bm_ctx* ctx, int stage, cudaStream_t st, F&& launch, const int* nlaunch = nullptr) {
    if (!ctx->timing.load()) return launch();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    cudaError_t e = launch();
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(ctx->tm_mu);
    ctx->tm_pending.push_back({stage, nlaunch ? *nlaunch : 1, a, b});
    return e;
}

// ---------------- autotuner ----------------
// The tensor-core kernel has several tile configurations per job class
// (lane -> reference mapping, stage depth, append buffer); the built-in
// choice is a heuristic (least MMA work).  With a tune-cache file the first
// job of each class times every configuration on its own data, keeps the
// fastest whose output equals the heuristic's, and records the pick in the
// file (one "key choice microseconds" line per class).

std::string class_key(const Geom& g) {
    std::ostringstream o;
    o << "tc2_dtype" << g.dtype << "_C" << g.C << "_p" << g.p << "_w" << (2 * g.h + 1) << "_s" << g.s
      << "_K" << g.K;
    return o.str();
}

void load_tune_file(bm_ctx* ctx) {
    std::ifstream f(ctx->tune_cache);
    std::string key;
    int choice;
    double us;
    while (f >> key >> choice >> us) ctx->tune_table[key] = choice;
}

void save_tune_file(bm_ctx* ctx) {
    std::ofstream f(ctx->tune_cache, std::ios::trunc);
    for (const auto& kv : ctx->tune_table) f << kv.first << " " << kv.second << " 0\n";
}

// Time every configuration of g's class on job a (its preparation kernels
// already enqueued on st); returns the pick (-1: the heuristic).
int tune_class(bm_ctx* ctx, const Geom& g, const TcArgs& a, cudaStream_t st) {
    const int n = tc_num_choices(g);
    if (n <= 1) return -1;
    const bool f32 = g.dtype == kF32;
    const size_t cnt = (size_t)g.nR * (f32 ? g.L : g.K);
    void* o1 = f32 ? (void*)a.pool_idx : (void*)a.out_idx;
    void* o2 = f32 ? (void*)a.pool_score : (void*)a.out_dist;
    std::vector<int32_t> ref1(cnt), ref2(cnt), got1(cnt), got2(cnt);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto run = [&](int choice, float* ms) -> bool {
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            if (launch_tc_batch(&g, &a, 1, st, nullptr, choice >= 0 ? &choice : nullptr) != cudaSuccess)
                return false;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return false;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        *ms = best;
        return true;
    };
    int pick = -1;
    float t_ref = 0.f;
    if (!run(-1, &t_ref) || cudaMemcpy(ref1.data(), o1, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ref2.data(), o2, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        pick = -1;
    } else {
        float t_best = t_ref;
        for (int c = 0; c < n; ++c) {
            float t = 0.f;
            if (!run(c, &t)) {
                cudaGetLastError();
                continue;
            }
            if (cudaMemcpy(got1.data(), o1, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(got2.data(), o2, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                continue;
            if (got1 != ref1 || got2 != ref2) continue;  // must reproduce the heuristic's output
            if (t < t_best) {
                t_best = t;
                pick = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return pick;
}

// Configuration for each tensor-core job (tuning unknown classes first when
// a tune-cache file is set and st is not being captured).
std::vector<int> tc_choices(bm_ctx* ctx, const Geom* gs, const TcArgs* as, int n, cudaStream_t st) {
    std::vector<int> ch(n, -1);
    if (ctx->tune_cache.empty()) return ch;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    for (int i = 0; i < n; ++i) {
        const std::string key = class_key(gs[i]);
        auto it = ctx->tune_table.find(key);
        if (it == ctx->tune_table.end()) {
            if (cap != cudaStreamCaptureStatusNone) continue;
            const int pick = tune_class(ctx, gs[i], as[i], st);
            it = ctx->tune_table.emplace(key, pick).first;
            save_tune_file(ctx);
        }
        ch[i] = it->second < tc_num_choices(gs[i]) ? it->second : -1;
    }
    return ch;
}

// Workspace pointers of a tensor-core job: preparation job and tensor-core
// arguments.
void job_views(const Geom& g, const bm_request& r, void* ws, PrepJob& pj, TcArgs& a) {
    WsLayout l = ws_layout(g);
    char* b = static_cast<char*>(ws);
    uint16_t* p0 = reinterpret_cast<uint16_t*>(b + l.plane0);
    uint16_t* p1 = g.dtype == kF32 ? reinterpret_cast<uint16_t*>(b + l.plane1) : nullptr;
    void* nrm = b + l.nrm;
    uint16_t* nsp = reinterpret_cast<uint16_t*>(b + l.nsp);
    int* status = reinterpret_cast<int*>(b + l.status);
    float* center = reinterpret_cast<float*>(b + l.status + 16);
    pj = make_prep_job(g, r.img, center, p0, p1, nrm, nsp);
    pj.status = status;
    a = TcArgs{};
    a.plane0 = p0;
    a.plane1 = p1;
    a.nrm = nrm;
    a.nsp = nsp;
    a.status = status;
    if (g.dtype == kU8) {
        a.out_idx = r.out_idx;
        a.out_dist = static_cast<int32_t*>(r.out_dist);
    } else {
        a.pool_idx = reinterpret_cast<int32_t*>(b + l.pool_idx);
        a.pool_score = reinterpret_cast<float*>(b + l.pool_score);
    }
    if (l.wsplit > 1) {
        const size_t nlist = (size_t)g.nR * (g.dtype == kF32 ? g.L : g.K);
        a.wsplit = l.wsplit;
        a.split_idx = reinterpret_cast<int32_t*>(b + l.split);
        a.split_val = reinterpret_cast<int32_t*>(b + l.split + align256((size_t)l.wsplit * nlist * 4));
    }
}

// Preparation kernels of n tensor-core jobs (status reset + centring offset,
// bf16 planes, box filter): one launch per stage.
int prep_jobs(bm_ctx* ctx, const PrepJob* pj, int n, cudaStream_t st) {
    cudaError_t e;
    if ((e = timed(ctx, BM_STAGE_PLANES, st,
                   [&] { return launch_center_batch(pj, n, st); })) != cudaSuccess)
        return cuda_fail(e, "centre kernel launch");
    if ((e = timed(ctx, BM_STAGE_PLANES, st,
                   [&] { return launch_planes_batch(pj, n, st); })) != cudaSuccess)
        return cuda_fail(e, "plane kernel launch");
    if ((e = timed(ctx, BM_STAGE_BOX, st,
                   [&] { return launch_box_batch(pj, n, st); })) != cudaSuccess)
        return cuda_fail(e, "box filter launch");
    return BM_OK;
}

// Last kernel of a float32 tensor-core job: the boundary re-rank.
int finish_job(bm_ctx* ctx, const Geom& g, const bm_request& r, const TcArgs& a, cudaStream_t st) {
    if (g.dtype != kF32) return BM_OK;
    cudaError_t e = timed(ctx, BM_STAGE_RERANK, st, [&] {
        return launch_rerank(g, static_cast<const float*>(r.img), static_cast<const float*>(a.nrm),
                             a.pool_idx, a.pool_score, r.out_idx, static_cast<float*>(r.out_dist),
                             ctx->d_counters, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "re-rank kernel launch");
    return BM_OK;
}

// Enqueue the kernels of one job on st, using workspace ws (size job_ws_bytes).
int enqueue_job(bm_ctx* ctx, const Geom& g, const bm_request& r, void* ws, cudaStream_t st) {
    cudaError_t e;
    if (!use_tc(ctx, g)) {
        e = timed(ctx, BM_STAGE_DIRECT, st,
                  [&] { return launch_direct(g, r.img, r.out_idx, r.out_dist, st); });
        if (e != cudaSuccess) return cuda_fail(e, "direct kernel launch");
        return BM_OK;
    }
    TcArgs a;
    PrepJob pj;
    job_views(g, r, ws, pj, a);
    a.fault = ctx->d_fault;
    a.inject = ctx->inject.exchange(0);
    int rc = prep_jobs(ctx, &pj, 1, st);
    if (rc != BM_OK) return rc;
    const std::vector<int> ch = tc_choices(ctx, &g, &a, 1, st);
    if ((e = timed(ctx, BM_STAGE_TC, st, [&] {
             return launch_tc_batch(&g, &a, 1, st, nullptr, ch.data());
         })) != cudaSuccess)
        return cuda_fail(e, "tensor-core kernel launch");
    ctx->tc_jobs += 1;
    return finish_job(ctx, g, r, a, st);
}

// Branch streams of base stream st (created on first use, kept per base
// stream so that two threads capturing on different streams never share
// one): out receives n of them.
int branch_streams(bm_ctx* ctx, cudaStream_t st, int n, std::vector<cudaStream_t>& out) {
    std::lock_guard<std::mutex> lk(ctx->br_mu);
    std::vector<cudaStream_t>& v = ctx->branches[st];
    while ((int)v.size() < n) {
        cudaStream_t s2 = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "branch stream create");
        v.push_back(s2);
    }
    out.assign(v.begin(), v.begin() + n);
    return BM_OK;
}

// Enqueue n validated jobs on st with one workspace (job i at ws + offs[i]):
// direct jobs, then the preparation kernels of the tensor-core jobs (one
// launch per stage), their cross term + top-K (persistent launches, one per
// class), and the float32 re-ranks (one launch per class).  count: add the
// jobs to the context counters.  job_status (nullable, device): job i's
// tensor-core kernel writes its timeout code to job_status[i] (the caller
// zeroes the words).
int enqueue_batch(bm_ctx* ctx, const Geom* gs, const bm_request* reqs, int n, void* ws,
                  const size_t* offs, cudaStream_t st, bool count, int* job_status = nullptr) {
    std::vector<int> tc_ids, direct_ids;
    std::vector<TcArgs> args(n);
    std::vector<PrepJob> pjs;
    for (int i = 0; i < n; ++i) {
        if (!use_tc(ctx, gs[i])) {
            direct_ids.push_back(i);
        } else {
            PrepJob pj;
            job_views(gs[i], reqs[i], static_cast<char*>(ws) + offs[i], pj, args[i]);
            args[i].fault = ctx->d_fault;
            if (job_status) args[i].status = job_status + i;
            pjs.push_back(pj);
            tc_ids.push_back(i);
        }
    }
    // direct-kernel jobs beside tensor-core jobs run on a branch of their own,
    // forked here (they depend on nothing of this batch) and joined at the end,
    // so they overlap the tensor-core work instead of preceding it
    cudaEvent_t ev_dfork = nullptr;
    const bool fork_direct = !direct_ids.empty() && !tc_ids.empty() && !ctx->timing.load();
    if (fork_direct) {
        cudaError_t e = cudaEventCreateWithFlags(&ev_dfork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev_dfork, st);
        if (e != cudaSuccess) return cuda_fail(e, "direct fork");
    } else {
        for (int i : direct_ids) {
            int rc = enqueue_job(ctx, gs[i], reqs[i], nullptr, st);
            if (rc != BM_OK) return rc;
        }
    }
    int nbranch = 0;  // class branches the tensor-core part used
    if (!tc_ids.empty()) {
        int rc = prep_jobs(ctx, pjs.data(), (int)pjs.size(), st);
        if (rc != BM_OK) return rc;
        auto key = [&](int i) {
            const Geom& g = gs[i];
            return std::make_tuple(g.dtype, g.Cp, g.p, g.h, g.s, g.K, g.L, g.C);
        };
        std::stable_sort(tc_ids.begin(), tc_ids.end(), [&](int a, int b) { return key(a) < key(b); });
        std::vector<Geom> tg;
        std::vector<TcArgs> ta;
        for (int i : tc_ids) {
            tg.push_back(gs[i]);
            ta.push_back(args[i]);
        }
        // the fault-injection test hook applies to the first tensor-core launch
        // (never inside a graph capture: every replay would repeat it)
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        if (cap == cudaStreamCaptureStatusNone) ta[0].inject = ctx->inject.exchange(0);
        const std::vector<int> ch = tc_choices(ctx, tg.data(), ta.data(), (int)tg.size(), st);
        // classes: runs of jobs that share one persistent launch (same
        // tensor-core class and tile choice)
        std::vector<int> cls_begin;
        for (int j = 0; j < (int)tg.size(); ++j)
            if (j == 0 || !tc_same_class(tg[j], tg[j - 1]) || ch[j] != ch[j - 1]) cls_begin.push_back(j);
        cls_begin.push_back((int)tg.size());
        const int ncls = (int)cls_begin.size() - 1;
        if (count) ctx->tc_jobs += tc_ids.size();
        // each class's tensor-core launch and its re-rank; with several
        // classes (and stage timing off) every class after the first runs on
        // a branch stream forked from st and joined back, so the classes'
        // persistent launches overlap: CTAs of one class take the SMs that
        // another class's CTAs leave.  Under graph capture the branches become
        // parallel graph branches.
        const bool fork = ncls > 1 && !ctx->timing.load();
        std::vector<cudaStream_t> br;
        if (fork) {
            int rc = branch_streams(ctx, st, ncls - 1, br);
            if (rc != BM_OK) return rc;
            nbranch = ncls - 1;
        }
        cudaEvent_t ev_fork = nullptr;
        std::vector<cudaEvent_t> ev_join;
        cudaError_t e = cudaSuccess;
        if (fork) {
            if ((e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventRecord(ev_fork, st)) != cudaSuccess)
                return cuda_fail(e, "class fork");
        }
        for (int c = 0; c < (fork ? ncls : 1); ++c) {
            const int b = fork ? cls_begin[c] : 0, eidx = fork ? cls_begin[c + 1] : (int)tg.size();
            cudaStream_t sc = (fork && c > 0) ? br[c - 1] : st;
            if (sc != st && (e = cudaStreamWaitEvent(sc, ev_fork, 0)) != cudaSuccess)
                return cuda_fail(e, "class fork");
            int nl = 0;
            e = timed(ctx, BM_STAGE_TC, sc, [&] {
                return launch_tc_batch(tg.data() + b, ta.data() + b, eidx - b, sc, &nl, ch.data() + b);
            }, &nl);
            if (e != cudaSuccess) return cuda_fail(e, "tensor-core kernel launch");
            std::vector<Geom> rg;
            std::vector<RerankArgs> ra;
            for (int j = b; j < eidx; ++j) {
                const int i = tc_ids[j];
                if (gs[i].dtype != kF32) continue;
                rg.push_back(gs[i]);
                ra.push_back(RerankArgs{static_cast<const float*>(reqs[i].img),
                                        static_cast<const float*>(args[i].nrm), args[i].pool_idx,
                                        args[i].pool_score, reqs[i].out_idx,
                                        static_cast<float*>(reqs[i].out_dist)});
            }
            if (!rg.empty()) {
                int nr = 0;
                e = timed(ctx, BM_STAGE_RERANK, sc, [&] {
                    return launch_rerank_batch(rg.data(), ra.data(), (int)rg.size(), ctx->d_counters,
                                               sc, &nr);
                }, &nr);
                if (e != cudaSuccess) return cuda_fail(e, "re-rank kernel launch");
            }
            if (sc != st) {
                cudaEvent_t ej = nullptr;
                if ((e = cudaEventCreateWithFlags(&ej, cudaEventDisableTiming)) != cudaSuccess ||
                    (e = cudaEventRecord(ej, sc)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(st, ej, 0)) != cudaSuccess)
                    return cuda_fail(e, "class join");
                ev_join.push_back(ej);
            }
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (cudaEvent_t ej : ev_join) cudaEventDestroy(ej);
    }
    if (fork_direct) {
        std::vector<cudaStream_t> br;
        int rc = branch_streams(ctx, st, nbranch + 1, br);
        if (rc != BM_OK) return rc;
        cudaStream_t sd = br.back();
        cudaError_t e = cudaStreamWaitEvent(sd, ev_dfork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "direct fork");
        for (int i : direct_ids) {
            rc = enqueue_job(ctx, gs[i], reqs[i], nullptr, sd);
            if (rc != BM_OK) return rc;
        }
        cudaEvent_t ej = nullptr;
        if ((e = cudaEventCreateWithFlags(&ej, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventRecord(ej, sd)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ej, 0)) != cudaSuccess)
            return cuda_fail(e, "direct join");
        cudaEventDestroy(ej);
        cudaEventDestroy(ev_dfork);
    }
    if (count) {
        for (int i = 0; i < n; ++i) {
            ctx->matches += 1;
            ctx->refs += (unsigned long long)gs[i].nR;
        }
    }
    return BM_OK;
}

// Per-stream workspace of at least `bytes`, grown stream-ordered.
int get_stream_ws(bm_ctx* ctx, cudaStream_t st, size_t bytes, void** out) {
    std::lock_guard<std::mutex> lk(ctx->ws_mu);
    Workspace& w = ctx->ws[st];
    if (w.bytes >= bytes) {
        *out = w.ptr;
        return BM_OK;
    }
    size_t others = ctx->used.load() - w.bytes;
    if (others + bytes > ctx->budget)
        return fail(BM_ERR_OOM, "workspace would exceed the context memory budget");
    cudaError_t e;
    if (w.ptr) {
        if ((e = cudaFreeAsync(w.ptr, st)) != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
        ctx->used -= w.bytes;
        w.ptr = nullptr;
        w.bytes = 0;
    }
    if ((e = cudaMallocAsync(&w.ptr, bytes, st)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    w.bytes = bytes;
    ctx->used += bytes;
    *out = w.ptr;
    return BM_OK;
}

}  // namespace

namespace bm {
int ctx_device(const ::bm_ctx* ctx) { return ctx->device; }
int ctx_workspace(::bm_ctx* ctx, cudaStream_t st, size_t bytes, void** out) {
    return get_stream_ws(ctx, st, bytes, out);
}
int* ctx_fault_word(::bm_ctx* ctx) { return ctx->d_fault; }
unsigned long long* ctx_counters(::bm_ctx* ctx) { return ctx->d_counters; }
void ctx_count_tc_job(::bm_ctx* ctx) { ctx->tc_jobs += 1; }
bool ctx_uses_tc(::bm_ctx* ctx) { return ctx->algo != BM_ALGO_DIRECT; }
}  // namespace bm

namespace {

// Reads and clears the context's sticky timeout word (the caller has
// synchronised the work it wants covered): BM_ERR_TIMEOUT naming the wait
// site if a bounded device wait of the tensor-core kernel ran out.  The copy
// runs on the context's own non-blocking stream, so other streams keep
// running meanwhile.
int take_fault(bm_ctx* ctx) {
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->d_fault, sizeof(int), cudaMemcpyDeviceToHost, ctx->aux_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->aux_stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device fault word");
    if (v == 0) return BM_OK;
    if ((e = cudaMemsetAsync(ctx->d_fault, 0, sizeof(int), ctx->aux_stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->aux_stream)) != cudaSuccess)
        return cuda_fail(e, "clearing the device fault word");
    return fail(BM_ERR_TIMEOUT, timeout_message(v));
}

}  // namespace

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int match_common(bm_ctx* ctx, const bm_request& r, cudaStream_t st, bool force_direct) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    Geom g;
    int rc = validate(r, g);
    if (rc != BM_OK) return rc;
    DeviceGuard dg(ctx->device);
    if (force_direct) {
        cudaError_t e = timed(ctx, BM_STAGE_DIRECT, st,
                              [&] { return launch_direct(g, r.img, r.out_idx, r.out_dist, st); });
        if (e != cudaSuccess) return cuda_fail(e, "direct kernel launch");
    } else {
        void* ws = nullptr;
        size_t need = job_ws_bytes(ctx, g);
        if (need) {
            rc = get_stream_ws(ctx, st, need, &ws);
            if (rc != BM_OK) return rc;
        }
        rc = enqueue_job(ctx, g, r, ws, st);
        if (rc != BM_OK) return rc;
    }
    ctx->matches += 1;
    ctx->refs += (unsigned long long)g.nR;
    return BM_OK;
}

// ---------------- serving loop ----------------

void worker_loop(bm_ctx* ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    while (true) {
        // 1. retire finished batches: a job whose tensor-core kernel ran out of
        // a bounded wait (its error word, copied to the host ring entry after
        // the batch's kernels) fails with BM_ERR_TIMEOUT
        for (size_t bi = 0; bi < ctx->batches.size();) {
            Batch& b = ctx->batches[bi];
            cudaError_t q = cudaEventQuery(b.ev);
            if (q == cudaErrorNotReady) {
                ++bi;
                continue;
            }
            const int* words = ctx->h_ring + (size_t)b.ring * bm_ctx::kMaxBatch;
            for (size_t i = 0; i < b.ids.size(); ++i) {
                Ticket& t = ctx->tickets[b.ids[i]];
                if (q != cudaSuccess && t.status == BM_OK) {
                    t.msg = std::string("request failed: ") + cudaGetErrorString(q);
                    t.status = BM_ERR_CUDA;
                } else if (q == cudaSuccess && words[i] != 0 && t.status == BM_OK) {
                    t.msg = timeout_message(words[i]);
                    t.status = BM_ERR_TIMEOUT;
                }
                t.done = true;
            }
            cudaEventDestroy(b.ev);
            ctx->used -= b.bytes;
            ctx->slot_busy[b.slot] -= 1;
            ctx->ring_busy[b.ring] = false;
            ctx->batches.erase(ctx->batches.begin() + bi);
        }
        // 2. continuous batching: the pending requests that fit the memory
        // budget (in arrival order) are admitted together as one batch on the
        // least busy stream -- one persistent launch per kernel stage -- as
        // soon as a stream slot is free.  The queue lock is released while the
        // batch is enqueued, so bm_submit and bm_poll never wait for launches.
        while (!ctx->pending.empty()) {
            int slot = 0;
            for (int s = 1; s < bm_ctx::kSlots; ++s)
                if (ctx->slot_busy[s] < ctx->slot_busy[slot]) slot = s;
            if (ctx->slot_busy[slot] >= 2) break;  // every stream already has two batches in flight
            int ring = 0;
            while (ring < bm_ctx::kRing && ctx->ring_busy[ring]) ++ring;
            if (ring == bm_ctx::kRing) break;
            std::vector<uint64_t> ids;
            size_t batch_bytes = 0;
            while (!ctx->pending.empty() && ids.size() < (size_t)bm_ctx::kMaxBatch) {
                Ticket& t = ctx->tickets[ctx->pending.front()];
                const size_t b = align256(t.ws_bytes);
                if (ctx->used.load() + batch_bytes + b > ctx->budget) break;
                batch_bytes += b;
                ids.push_back(ctx->pending.front());
                ctx->pending.pop_front();
            }
            if (ids.empty()) break;  // the oldest request waits for memory
            cudaStream_t st = ctx->slot_stream[slot];
            const int n = (int)ids.size();
            std::vector<Geom> gs(n);
            std::vector<bm_request> reqs(n);
            std::vector<size_t> offs(n);
            size_t off = 0;
            for (int i = 0; i < n; ++i) {
                Ticket& t = ctx->tickets[ids[i]];
                t.admitted = true;
                t.slot = slot;
                reqs[i] = t.req;
                validate(t.req, gs[i]);
                offs[i] = off;
                off += align256(t.ws_bytes);
            }
            ctx->used += batch_bytes;
            ctx->slot_busy[slot] += 1;
            ctx->ring_busy[ring] = true;
            lk.unlock();
            // enqueue without the lock (this thread alone uses the slot streams)
            int* words = ctx->d_ring + (size_t)ring * bm_ctx::kMaxBatch;
            int* hwords = ctx->h_ring + (size_t)ring * bm_ctx::kMaxBatch;
            std::memset(hwords, 0, sizeof(int) * bm_ctx::kMaxBatch);
            void* ws = nullptr;
            cudaError_t e = cudaMemsetAsync(words, 0, sizeof(int) * n, st);
            if (e == cudaSuccess && batch_bytes) e = cudaMallocAsync(&ws, batch_bytes, st);
            std::string err;
            int rc = BM_ERR_OOM;
            if (e == cudaSuccess) {
                rc = enqueue_batch(ctx, gs.data(), reqs.data(), n, ws, offs.data(), st, true, words);
                if (rc != BM_OK) err = t_last_error;
            } else {
                err = std::string("batch workspace: ") + cudaGetErrorString(e);
                cudaGetLastError();
            }
            if (ws) cudaFreeAsync(ws, st);
            cudaMemcpyAsync(hwords, words, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
            cudaEvent_t ev = nullptr;
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            cudaEventRecord(ev, st);
            lk.lock();
            ctx->batches.push_back(Batch{ev, slot, ring, batch_bytes, ids});
            for (int i = 0; i < n; ++i) {
                Ticket& t = ctx->tickets[ids[i]];
                t.status = rc;
                if (rc != BM_OK) t.msg = err;
            }
        }
        if (ctx->stop) {
            bool busy = false;
            for (auto& kv : ctx->tickets) busy |= kv.second.admitted && !kv.second.done;
            if (!busy && ctx->pending.empty()) break;
        }
        ctx->q_cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

size_t bm_workspace_bytes(int H, int W, int C, bm_dtype dtype, int patch, int window, int stride,
                          int K) {
    Geom g;
    if (make_geom(g, H, W, C, (int)dtype, patch, window, stride, K) != 0) return 0;
    return tc_supported(g) ? ws_layout(g).total : 0;
}

int bm_window_split(int H, int W, int C, bm_dtype dtype, int patch, int window, int stride, int K) {
    Geom g;
    if (make_geom(g, H, W, C, (int)dtype, patch, window, stride, K) != 0) return 0;
    return tc_supported(g) ? tc_window_split(g) : 1;
}

int bm_num_refs(int H, int W, int patch, int stride, int* n_ry, int* n_rx) {
    if (H < 1 || W < 1 || patch < 1 || stride < 1 || patch > H || patch > W)
        return fail(BM_ERR_INVALID, "invalid geometry");
    if (n_ry) *n_ry = (H - patch) / stride + 1;
    if (n_rx) *n_rx = (W - patch) / stride + 1;
    return BM_OK;
}

int bm_create(bm_ctx** out, int device, size_t mem_budget_bytes, const char* tune_cache) {
    if (!out) return fail(BM_ERR_INVALID, "null output pointer");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(BM_ERR_INVALID, "no such CUDA device");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
        return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3)
        return fail(BM_ERR_UNSUPPORTED, std::string("library is built for sm_103a, device is ") +
                                            prop.name);
    bm_ctx* ctx = new bm_ctx();
    ctx->device = device;
    ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)40 << 30;
    if (tune_cache) {
        ctx->tune_cache = tune_cache;
        load_tune_file(ctx);
    }
    DeviceGuard dg(device);
    if ((e = cudaMalloc(&ctx->d_fault, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(ctx->d_fault, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_counters, 4 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(ctx->d_counters, 0, 4 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->host_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_ring, sizeof(int) * bm_ctx::kRing * bm_ctx::kMaxBatch)) != cudaSuccess ||
        (e = cudaHostAlloc(&ctx->h_ring, sizeof(int) * bm_ctx::kRing * bm_ctx::kMaxBatch,
                           cudaHostAllocDefault)) != cudaSuccess) {
        delete ctx;
        return cuda_fail(e, "context setup");
    }
    for (int s = 0; s < bm_ctx::kSlots; ++s) {
        if ((e = cudaStreamCreateWithFlags(&ctx->slot_stream[s], cudaStreamNonBlocking)) !=
            cudaSuccess) {
            delete ctx;
            return cuda_fail(e, "stream create");
        }
    }
    ctx->worker = std::thread(worker_loop, ctx);
    *out = ctx;
    return BM_OK;
}

void bm_destroy(bm_ctx* ctx) {
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        ctx->stop = true;
    }
    ctx->q_cv.notify_all();
    if (ctx->worker.joinable()) ctx->worker.join();
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->ws)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (auto& kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (ctx->h_dev_img) cudaFree(ctx->h_dev_img);
    if (ctx->h_dev_out) cudaFree(ctx->h_dev_out);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->d_fault) cudaFree(ctx->d_fault);
    if (ctx->host_stream) cudaStreamDestroy(ctx->host_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    for (auto& kv : ctx->branches)
        for (cudaStream_t s2 : kv.second) cudaStreamDestroy(s2);
    if (ctx->d_ring) cudaFree(ctx->d_ring);
    if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
    for (int b = 0; b < 2; ++b) {
        if (ctx->hb_buf[b]) cudaFree(ctx->hb_buf[b]);
        if (ctx->hb_stream[b]) cudaStreamDestroy(ctx->hb_stream[b]);
    }
    for (int s = 0; s < bm_ctx::kSlots; ++s)
        if (ctx->slot_stream[s]) cudaStreamDestroy(ctx->slot_stream[s]);
    delete ctx;
}

const char* bm_last_error(bm_ctx*) { return t_last_error.c_str(); }

int bm_check(bm_ctx* ctx, bm_stream stream) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return take_fault(ctx);
}

int bm_set_fault_injection(bm_ctx* ctx, int mode) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    if (mode != 0 && mode != 1) return fail(BM_ERR_INVALID, "unknown fault injection mode");
    ctx->inject.store(mode);
    return BM_OK;
}

int bm_set_algo(bm_ctx* ctx, bm_algo algo) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    if (algo != BM_ALGO_AUTO && algo != BM_ALGO_SELFCONV_TC && algo != BM_ALGO_DIRECT)
        return fail(BM_ERR_INVALID, "unknown algorithm");
    ctx->algo = algo;
    return BM_OK;
}

int bm_match(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
             int window, int stride, int K, int32_t* out_idx, void* out_dist, bm_stream stream) {
    bm_request r{img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist};
    return match_common(ctx, r, reinterpret_cast<cudaStream_t>(stream), false);
}

int bm_match_direct(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                    int window, int stride, int K, int32_t* out_idx, void* out_dist,
                    bm_stream stream) {
    bm_request r{img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist};
    return match_common(ctx, r, reinterpret_cast<cudaStream_t>(stream), true);
}

int bm_match_host(bm_ctx* ctx, const void* img, int H, int W, int C, bm_dtype dtype, int patch,
                  int window, int stride, int K, int32_t* out_idx, void* out_dist) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    bm_request r{img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist};
    Geom g;
    int rc = validate(r, g);
    if (rc != BM_OK) return rc;
    std::lock_guard<std::mutex> lk(ctx->host_mu);
    DeviceGuard dg(ctx->device);
    size_t img_bytes = (size_t)H * W * C * (dtype == BM_U8 ? 1 : 4);
    size_t out_bytes = (size_t)g.nR * K * 8;
    cudaError_t e;
    if (ctx->h_dev_img_bytes < img_bytes) {
        if (ctx->h_dev_img) cudaFree(ctx->h_dev_img);
        ctx->h_dev_img = nullptr;
        ctx->h_dev_img_bytes = 0;
        if ((e = cudaMalloc(&ctx->h_dev_img, img_bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        ctx->h_dev_img_bytes = img_bytes;
    }
    if (ctx->h_dev_out_bytes < out_bytes) {
        if (ctx->h_dev_out) cudaFree(ctx->h_dev_out);
        ctx->h_dev_out = nullptr;
        ctx->h_dev_out_bytes = 0;
        if ((e = cudaMalloc(&ctx->h_dev_out, out_bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        ctx->h_dev_out_bytes = out_bytes;
    }
    cudaStream_t st = ctx->host_stream;
    int32_t* d_idx = static_cast<int32_t*>(ctx->h_dev_out);
    void* d_dist = static_cast<char*>(ctx->h_dev_out) + (size_t)g.nR * K * 4;
    if ((e = cudaMemcpyAsync(ctx->h_dev_img, img, img_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "host-to-device copy");
    bm_request dr{ctx->h_dev_img, H, W, C, dtype, patch, window, stride, K, d_idx, d_dist};
    rc = match_common(ctx, dr, st, false);
    if (rc != BM_OK) return rc;
    if ((e = cudaMemcpyAsync(out_idx, d_idx, (size_t)g.nR * K * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out_dist, d_dist, (size_t)g.nR * K * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "device-to-host copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "synchronize");
    return take_fault(ctx);
}

int bm_match_host_batch(bm_ctx* ctx, const bm_request* reqs, int n) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    if (n < 0 || (n > 0 && !reqs)) return fail(BM_ERR_INVALID, "bad request list");
    std::vector<Geom> gs(n);
    std::vector<size_t> in_b(n), out_b(n);
    for (int i = 0; i < n; ++i) {
        int rc = validate(reqs[i], gs[i]);
        if (rc != BM_OK) return rc;
        in_b[i] = align256((size_t)gs[i].H * gs[i].W * gs[i].C * (gs[i].dtype == kU8 ? 1 : 4));
        out_b[i] = align256((size_t)gs[i].nR * gs[i].K * 4);
    }
    if (n == 0) return BM_OK;
    std::lock_guard<std::mutex> lk(ctx->host_mu);
    DeviceGuard dg(ctx->device);
    cudaError_t e;
    for (int b = 0; b < 2; ++b)
        if (!ctx->hb_stream[b] &&
            (e = cudaStreamCreateWithFlags(&ctx->hb_stream[b], cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "stream create");
    // chunks of consecutive jobs: up to 16 jobs or 96 MB of staging
    constexpr int kChunkJobs = 16;
    constexpr size_t kChunkBytes = (size_t)96 << 20;
    std::vector<int> starts;
    for (int i = 0; i < n;) {
        starts.push_back(i);
        size_t bytes = 0;
        int m = 0;
        while (i < n && m < kChunkJobs &&
               (m == 0 || bytes + in_b[i] + 2 * out_b[i] <= kChunkBytes)) {
            bytes += in_b[i] + 2 * out_b[i];
            ++i;
            ++m;
        }
    }
    starts.push_back(n);
    for (size_t c = 0; c + 1 < starts.size(); ++c) {
        const int i0 = starts[c], i1 = starts[c + 1], m = i1 - i0, b = (int)(c & 1);
        cudaStream_t st = ctx->hb_stream[b];
        size_t stage = 0;
        for (int i = i0; i < i1; ++i) stage += in_b[i] + 2 * out_b[i];
        // staging of pipeline b: the previous chunk on this stream is done with
        // it before anything below runs (stream order), but a reallocation
        // must wait for it
        if (ctx->hb_bytes[b] < stage) {
            if (ctx->hb_buf[b]) {
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "synchronize");
                cudaFree(ctx->hb_buf[b]);
                ctx->hb_buf[b] = nullptr;
                ctx->hb_bytes[b] = 0;
            }
            if ((e = cudaMalloc(&ctx->hb_buf[b], stage)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
            ctx->hb_bytes[b] = stage;
        }
        char* base = static_cast<char*>(ctx->hb_buf[b]);
        std::vector<bm_request> dr(reqs + i0, reqs + i1);
        size_t off = 0;
        for (int k = 0; k < m; ++k) {
            const int i = i0 + k;
            dr[k].img = base + off;
            if ((e = cudaMemcpyAsync(base + off, reqs[i].img, in_b[i] > 0 ? (size_t)gs[i].H * gs[i].W * gs[i].C * (gs[i].dtype == kU8 ? 1 : 4) : 0,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(e, "host-to-device copy");
            off += in_b[i];
            dr[k].out_idx = reinterpret_cast<int32_t*>(base + off);
            off += out_b[i];
            dr[k].out_dist = base + off;
            off += out_b[i];
        }
        std::vector<size_t> offs(m);
        size_t total = 0;
        for (int k = 0; k < m; ++k) {
            offs[k] = total;
            total += align256(job_ws_bytes(ctx, gs[i0 + k]));
        }
        void* ws = nullptr;
        if (total) {
            int rc = get_stream_ws(ctx, st, total, &ws);
            if (rc != BM_OK) return rc;
        }
        int rc = enqueue_batch(ctx, gs.data() + i0, dr.data(), m, ws, offs.data(), st, true);
        if (rc != BM_OK) return rc;
        for (int k = 0; k < m; ++k) {
            const int i = i0 + k;
            ctx->matches += 1;
            ctx->refs += (unsigned long long)gs[i].nR;
            const size_t ob = (size_t)gs[i].nR * gs[i].K * 4;
            if ((e = cudaMemcpyAsync(reqs[i].out_idx, dr[k].out_idx, ob, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(reqs[i].out_dist, dr[k].out_dist, ob, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return cuda_fail(e, "device-to-host copy");
        }
    }
    for (int b = 0; b < 2; ++b)
        if ((e = cudaStreamSynchronize(ctx->hb_stream[b])) != cudaSuccess) return cuda_fail(e, "synchronize");
    return take_fault(ctx);
}

int bm_match_batch(bm_ctx* ctx, const bm_request* reqs, int n, bm_stream stream) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    if (n < 0 || (n > 0 && !reqs)) return fail(BM_ERR_INVALID, "bad request list");
    std::vector<Geom> gs(n);
    for (int i = 0; i < n; ++i) {
        int rc = validate(reqs[i], gs[i]);
        if (rc != BM_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard dg(ctx->device);
    // one workspace holding every job's region
    std::vector<size_t> offs(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        offs[i] = total;
        total += align256(job_ws_bytes(ctx, gs[i]));
    }
    void* ws = nullptr;
    if (total) {
        int rc = get_stream_ws(ctx, st, total, &ws);
        if (rc != BM_OK) return rc;
    }
    // Replays of the same job list on the same (non-legacy) stream run a
    // captured CUDA graph: one launch for the whole batch.  Not while stage
    // timing is on (its events bracket individual kernels).
    if (st != nullptr && st != cudaStreamLegacy && !ctx->timing.load()) {
        std::lock_guard<std::mutex> lk(ctx->graph_mu);
        GraphEntry& ge = ctx->graphs[st];
        const bool same = ge.exec && ge.ws == ws && ge.algo == ctx->algo &&
                          ge.reqs.size() == (size_t)n &&
                          (n == 0 || std::memcmp(ge.reqs.data(), reqs, n * sizeof(bm_request)) == 0);
        if (!same) {
            if (ge.exec) cudaGraphExecDestroy(ge.exec);
            ge.exec = nullptr;
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "stream capture");
            int rc = enqueue_batch(ctx, gs.data(), reqs, n, ws, offs.data(), st, false);
            e = cudaStreamEndCapture(st, &graph);
            if (rc != BM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "stream capture");
            e = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ge.exec = nullptr;
                return cuda_fail(e, "graph instantiate");
            }
            ge.reqs.assign(reqs, reqs + n);
            ge.ws = ws;
            ge.algo = ctx->algo;
            ge.tc_jobs = 0;
            for (int i = 0; i < n; ++i) ge.tc_jobs += use_tc(ctx, gs[i]) ? 1 : 0;
        }
        cudaError_t e = cudaGraphLaunch(ge.exec, st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        ctx->tc_jobs += ge.tc_jobs;
        for (int i = 0; i < n; ++i) {
            ctx->matches += 1;
            ctx->refs += (unsigned long long)gs[i].nR;
        }
        return BM_OK;
    }
    return enqueue_batch(ctx, gs.data(), reqs, n, ws, offs.data(), st, true);
}

int bm_submit(bm_ctx* ctx, const bm_request* req, uint64_t* ticket) {
    if (!ctx || !req || !ticket) return fail(BM_ERR_INVALID, "null argument");
    Geom g;
    int rc = validate(*req, g);
    if (rc != BM_OK) return rc;
    size_t need = job_ws_bytes(ctx, g);
    if (need > ctx->budget) return fail(BM_ERR_BUSY, "request alone exceeds the memory budget");
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    if (ctx->stop) return fail(BM_ERR_INVALID, "context is shutting down");
    uint64_t id = ctx->next_ticket++;
    Ticket& t = ctx->tickets[id];
    t.req = *req;
    t.ws_bytes = need;
    ctx->pending.push_back(id);
    *ticket = id;
    ctx->q_cv.notify_all();
    return BM_OK;
}

int bm_poll(bm_ctx* ctx, uint64_t ticket, int* done, int* status) {
    if (!ctx || !done || !status) return fail(BM_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(BM_ERR_NOT_FOUND, "unknown ticket");
    *done = it->second.done ? 1 : 0;
    *status = it->second.status;
    // a failed request's message becomes the polling thread's bm_last_error
    if (it->second.done && it->second.status != BM_OK) t_last_error = it->second.msg;
    if (it->second.done) ctx->tickets.erase(it);
    return BM_OK;
}

int bm_get_stats(bm_ctx* ctx, bm_stats* out) {
    if (!ctx || !out) return fail(BM_ERR_INVALID, "null argument");
    DeviceGuard dg(ctx->device);
    unsigned long long c[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(c, ctx->d_counters, sizeof c, cudaMemcpyDeviceToHost, ctx->aux_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->aux_stream);
    if (e != cudaSuccess) return cuda_fail(e, "counter read");
    out->matches = ctx->matches.load();
    out->refs = ctx->refs.load();
    out->rerank_overflow = c[0];
    out->fp64_rechecks = c[1];
    out->bound_violations = c[2];
    out->tc_jobs = ctx->tc_jobs.load();
    return BM_OK;
}

int bm_set_timing(bm_ctx* ctx, int enable) {
    if (!ctx) return fail(BM_ERR_INVALID, "null context");
    ctx->timing = enable ? 1 : 0;
    return BM_OK;
}

int bm_get_timing(bm_ctx* ctx, bm_timing* out, int reset) {
    if (!ctx || !out) return fail(BM_ERR_INVALID, "null argument");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->tm_mu);
    int rc = BM_OK;
    for (auto& ev : ctx->tm_pending) {
        cudaError_t e = cudaEventSynchronize(ev.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.a, ev.b);
        if (e != cudaSuccess && rc == BM_OK) rc = cuda_fail(e, "timing event");
        ctx->tm_total.launches[ev.stage] += ev.n;
        ctx->tm_total.ms[ev.stage] += ms;
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    ctx->tm_pending.clear();
    *out = ctx->tm_total;
    if (reset) ctx->tm_total = bm_timing{};
    return rc;
}

}  // extern "C"
