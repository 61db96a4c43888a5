// C ABI of the library (declared in include/rbs.h): argument checks, the
// per-(device, stream) workspace, host/device staging, and the solver driver
// that enqueues iterations and watches the device-resident stop flag.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "launch.h"

namespace rbs {
namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RBS_ENOMEM : RBS_ECUDA;
}
#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ---- knobs -------------------------------------------------------------------------
std::atomic<int64_t> p_exdot_grid{0}, p_exdot_block{0}, p_exdot_window{0}, p_spmv_block{0},
    p_vec_grid{0}, p_vec_block{0}, p_check_every{0}, p_spmv_mode{0}, p_carveout{75}, p_test_stall{0};

std::atomic<int64_t> *param_slot(const char *name) {
    if (!name) return nullptr;
    if (!strcmp(name, "exdot.grid")) return &p_exdot_grid;
    if (!strcmp(name, "exdot.block")) return &p_exdot_block;
    if (!strcmp(name, "exdot.window")) return &p_exdot_window;
    if (!strcmp(name, "spmv.block")) return &p_spmv_block;
    if (!strcmp(name, "vec.grid")) return &p_vec_grid;
    if (!strcmp(name, "vec.block")) return &p_vec_block;
    if (!strcmp(name, "solve.check_every")) return &p_check_every;
    if (!strcmp(name, "spmv.mode")) return &p_spmv_mode;
    if (!strcmp(name, "smem.carveout")) return &p_carveout;
    if (!strcmp(name, "test.stall_staging")) return &p_test_stall;
    return nullptr;
}

// SpMV row schedule: knob spmv.mode 1 (one thread per row), 2 (warp-staged,
// short spans) or 3 (warp-staged, long spans); 0 picks the staging from the
// average row length (long spans above 8 nonzeros per row).
int spmv_mode_for(int64_t n, int64_t nnz) {
    const int64_t m = p_spmv_mode.load();
    int mode = (n > 0 && nnz > 8 * n) ? SPMV_MODE_LONG : SPMV_MODE_SHORT;
    if (m == SPMV_MODE_ROW || m == SPMV_MODE_SHORT || m == SPMV_MODE_LONG) mode = (int)m;
    return mode | (p_test_stall.load() ? SPMV_TEST_STALL : 0);
}

int block_of(int64_t v, int def) {
    if (v <= 0) return def;
    int b = (int)(v > 256 ? 256 : v);
    b = (b / 32) * 32;
    return b < 32 ? 32 : b;
}

// ---- workspace ----------------------------------------------------------------------
struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

// Graph capture (graph_loop) runs in whichever thread calls a solve, and the
// serving runtime runs several such threads. cudaMalloc, cudaFree and device-
// wide synchronisation in one thread must not overlap a capture in another,
// so the library's own calls of that kind and its captures take this lock.
std::mutex g_cap_mu;

cudaError_t ensure(Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return cudaSuccess;
    std::lock_guard<std::mutex> cap(g_cap_mu);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.cap = bytes;
    return e;
}

// A pinned host buffer of at least `bytes` (contents not kept on growth).
cudaError_t ensure_host(Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return cudaSuccess;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMallocHost(&b.p, bytes);
    if (e == cudaSuccess) b.cap = bytes;
    return e;
}

constexpr int NVEC = 18;
constexpr int NFLAGS = 64;

struct Workspace {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    DotScratch *g = nullptr;
    SolverState *st = nullptr;
    SolverState *h_st = nullptr;
    int32_t *h_flags = nullptr;
    double *h_out = nullptr;
    double *d_out = nullptr;
    unsigned *h_err = nullptr;
    Buf vec, hist, stage[8];
    Buf batch_work, batch_hist, batch_sys, batch_order, batch_out, batch_queue;
    Buf step_ctx, step_state, step_scr, step_tasks;  // the stepped batch schedule
    std::vector<cudaEvent_t> evpool;
    std::vector<cudaEvent_t> ev_chunk;
    // graph loop: one iteration captured as the body of a conditional WHILE node
    cudaStream_t cap = nullptr;
    // the stepped batch: a second stream for the pipelined systems' steps, its
    // fork/join events, and pinned copies of the task list and the states
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Buf h_tasks, h_states;  // pinned (cudaMallocHost)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string graph_key;
    // batched solve: the per-batch launches captured once a system set and
    // schedule repeats (batch_seen: the previous call's key, not captured yet)
    cudaGraphExec_t batch_exec = nullptr;
    std::string batch_key, batch_seen;
    std::mutex mu;
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Workspace *> g_ws;

int ws_get(cudaStream_t s, Workspace **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) {
        *out = it->second;
        return RBS_OK;
    }
    std::lock_guard<std::mutex> cap(g_cap_mu);
    Workspace *w = new Workspace();
    w->dev = dev;
    w->stream = s;
    cudaError_t e = cudaDeviceGetAttribute(&w->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&w->g, sizeof(DotScratch));
    if (e == cudaSuccess) e = cudaMemset(w->g, 0, sizeof(DotScratch));
    if (e == cudaSuccess) e = cudaMalloc(&w->st, sizeof(SolverState));
    if (e == cudaSuccess) e = cudaMalloc(&w->d_out, KMAX * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&w->h_st, sizeof(SolverState));
    if (e == cudaSuccess) e = cudaMallocHost(&w->h_flags, NFLAGS * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&w->h_out, KMAX * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&w->h_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete w;
        return cuda_fail(e, "workspace creation");
    }
    g_ws[key] = w;
    *out = w;
    return RBS_OK;
}

void ws_free(Workspace *w) {
    std::lock_guard<std::mutex> cap(g_cap_mu);
    cudaSetDevice(w->dev);
    if (w->stream) cudaStreamSynchronize(w->stream);
    else cudaDeviceSynchronize();
    cudaFree(w->g);
    cudaFree(w->st);
    cudaFree(w->d_out);
    cudaFreeHost(w->h_st);
    cudaFreeHost(w->h_flags);
    cudaFreeHost(w->h_out);
    cudaFreeHost(w->h_err);
    cudaFree(w->vec.p);
    cudaFree(w->hist.p);
    for (Buf *b : {&w->batch_work, &w->batch_hist, &w->batch_sys, &w->batch_order, &w->batch_out,
                   &w->batch_queue, &w->step_ctx, &w->step_state, &w->step_scr, &w->step_tasks})
        cudaFree(b->p);
    for (auto &b : w->stage) cudaFree(b.p);
    for (auto e : w->evpool) cudaEventDestroy(e);
    for (auto e : w->ev_chunk) cudaEventDestroy(e);
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->graph) cudaGraphDestroy(w->graph);
    if (w->batch_exec) cudaGraphExecDestroy(w->batch_exec);
    if (w->cap) cudaStreamDestroy(w->cap);
    if (w->side) cudaStreamDestroy(w->side);
    if (w->ev_fork) cudaEventDestroy(w->ev_fork);
    if (w->ev_join) cudaEventDestroy(w->ev_join);
    if (w->h_tasks.p) cudaFreeHost(w->h_tasks.p);
    if (w->h_states.p) cudaFreeHost(w->h_states.p);
    delete w;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of a caller buffer: the pointer itself, or a staged copy
int to_device(Workspace *w, int slot, const void *p, size_t bytes, const void **out) {
    if (!p || bytes == 0 || is_device_ptr(p)) {
        *out = p;
        return RBS_OK;
    }
    CK(ensure(w->stage[slot], bytes));
    CK(cudaMemcpyAsync(w->stage[slot].p, p, bytes, cudaMemcpyHostToDevice, w->stream));
    *out = w->stage[slot].p;
    return RBS_OK;
}

int read_err(Workspace *w, unsigned *err) {
    CK(cudaMemcpyAsync(w->h_err, &w->g->err, sizeof(unsigned), cudaMemcpyDeviceToHost, w->stream));
    CK(cudaMemsetAsync(&w->g->err, 0, sizeof(unsigned), w->stream));
    CK(cudaStreamSynchronize(w->stream));
    *err = *w->h_err;
    return RBS_OK;
}

Cfg grid_for(Workspace *w, int64_t items, int block, int per_sm) {
    Cfg c;
    c.block = block;
    int64_t need = (items + block - 1) / block;
    int64_t cap = (int64_t)w->sms * per_sm;
    c.grid = (int)(need < 1 ? 1 : (need < cap ? need : cap));
    return c;
}

// Exact-dot launch shape: a persistent grid of whole waves (blocks_per_sm
// resident blocks on every SM), and never more than 2^20 products per thread
// per launch (the register window's headroom).
Cfg persistent_cfg(Workspace *w, int64_t n, int blocks_per_sm, int block) {
    Cfg c;
    c.block = block;
    int64_t g = p_exdot_grid.load();
    if (g <= 0) {
        int64_t need = (n + 2LL * c.block - 1) / (2LL * c.block);
        int64_t cap = (int64_t)w->sms * blocks_per_sm;
        g = need < 1 ? 1 : (need < cap ? need : cap);
    }
    int64_t minimum = (n + ((int64_t)c.block << 20) - 1) / ((int64_t)c.block << 20);
    if (g < minimum) g = minimum;
    if (g > 0x7fffffff) g = 0x7fffffff;
    c.grid = (int)g;
    return c;
}
Cfg exdot_cfg(Workspace *w, int64_t n, int k, int window) {
    const int block = block_of(p_exdot_block.load(), 256);
    return persistent_cfg(w, n, exdot_blocks_per_sm(k, window, block, n), block);
}

// Shared-memory carveout of the staging kernels. Measured on GB300 (Poisson
// 256^3): 60-75 % of the unified L1/shared storage is best -- enough shared
// memory for three 256-thread blocks per SM while L1 keeps the SpMV's x
// gathers; the maximum split costs about 5 % (25 % with a third staging
// buffer per warp), a small one halves throughput.
int carveout_param() {
    const int64_t c = p_carveout.load();
    return (c >= 0 && c <= 100) ? (int)c : -1;
}

int window_param() {
    int64_t q = p_exdot_window.load();
    return (q == 1 || q == 2 || q == 4) ? (int)q : 4;
}

// Per-kernel CUDA events. Kernels enqueued back to back share events: a
// kernel's start is the previous kernel's end, so each launch records one
// event; gap() marks other work in between (the next start is recorded anew).
// Each record carries the loop iteration it belongs to (-1: set-up) and its
// position within that iteration's launches.
struct EventTimer : KernelTimer {
    struct Rec {
        int kind, iter, slot;
        cudaEvent_t a, b;
    };
    Workspace *w;
    std::vector<Rec> rec;
    size_t used = 0;
    cudaEvent_t last_end = nullptr;
    cudaError_t err = cudaSuccess;
    int iter = -1, slot = 0;
    explicit EventTimer(Workspace *ws) : w(ws) {}
    cudaEvent_t take() {
        if (used == w->evpool.size()) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) {
                err = r;
                return nullptr;
            }
            w->evpool.push_back(e);
        }
        return w->evpool[used++];
    }
    void begin_iteration(int j) {
        iter = j;
        slot = 0;
    }
    void before(int kind) override {
        cudaEvent_t a = last_end;
        if (!a) {
            a = take();
            if (!a) return;
            cudaEventRecord(a, w->stream);
        }
        rec.push_back({kind, iter, slot++, a, nullptr});
    }
    void after(int kind) override {
        (void)kind;
        cudaEvent_t b = take();
        last_end = nullptr;
        if (!b || rec.empty()) return;
        cudaEventRecord(b, w->stream);
        rec.back().b = b;
        last_end = b;
    }
    void gap() override { last_end = nullptr; }
};

// Build (or reuse) the executable graph whose WHILE node replays one solver
// iteration until the device stop flag is set. Kernel arguments are baked in,
// so the graph is keyed by every launch argument; device scalars (tol, maxit)
// are not arguments and may change between solves.
int graph_loop(Workspace *w, const SolverArgs &a, int variant) {
    std::string key((const char *)&a, sizeof a);
    key.append((const char *)&variant, sizeof variant);
    if (!(w->exec && key == w->graph_key)) {
        std::lock_guard<std::mutex> cap(g_cap_mu);
        if (w->exec) cudaGraphExecDestroy(w->exec);
        if (w->graph) cudaGraphDestroy(w->graph);
        w->exec = nullptr;
        w->graph = nullptr;
        w->graph_key.clear();
        if (!w->cap) CK(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
        cudaGraph_t g;
        CK(cudaGraphCreate(&g, 0));
        w->graph = g;
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        CK(cudaStreamBeginCaptureToGraph(w->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = solver_iteration(a, variant, w->cap, nullptr);
        cudaError_t e2 = launch_set_cond(h, a.st, w->cap);
        cudaGraph_t out = nullptr;
        cudaError_t e3 = cudaStreamEndCapture(w->cap, &out);
        if (e1 != cudaSuccess) return cuda_fail(e1, "capture of the iteration");
        if (e2 != cudaSuccess) return cuda_fail(e2, "capture of the loop condition");
        if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamEndCapture");
        cudaGraphExec_t ex;
        CK(cudaGraphInstantiate(&ex, g, 0));
        w->exec = ex;
        w->graph_key = key;
    }
    CK(cudaGraphLaunch(w->exec, w->stream));
    return RBS_OK;
}

}  // namespace

int set_error(int code, const char *msg) { return fail(code, msg); }

void release_stream_workspace(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    Workspace *w = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find(std::make_pair(dev, s));
        if (it == g_ws.end()) return;
        w = it->second;
        g_ws.erase(it);
    }
    ws_free(w);
}

}  // namespace rbs

using namespace rbs;

extern "C" {

const char *rbs_version(void) { return "rbs 0.1 (sm_103a)"; }

const char *rbs_last_error(void) { return g_err.c_str(); }

int rbs_set_param(const char *name, int64_t value) {
    auto *s = param_slot(name);
    if (!s) return fail(RBS_EINVAL, std::string("unknown parameter ") + (name ? name : "(null)"));
    s->store(value);
    return RBS_OK;
}

int64_t rbs_get_param(const char *name) {
    auto *s = param_slot(name);
    return s ? s->load() : -1;
}

int rbs_release(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev0 = 0;
    cudaGetDevice(&dev0);
    for (auto &kv : g_ws) ws_free(kv.second);
    g_ws.clear();
    cudaSetDevice(dev0);
    return RBS_OK;
}

int rbs_stream_status(void *stream) {
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    unsigned err = 0;
    rc = read_err(w, &err);
    if (rc) return rc;
    if (err & 4u) return fail(RBS_ETIMEOUT, "a bounded wait on an asynchronous copy expired");
    if (err) return fail(RBS_EINVAL, "a kernel met an out-of-range CSR index");
    return RBS_OK;
}

static int exdot_common(int k, const double *const *xs, const double *const *ys, int64_t n, double *out,
                        void *stream) {
    if (k < 1 || k > KMAX) return fail(RBS_EINVAL, "k must be in 1..6");
    if (n < 0) return fail(RBS_EINVAL, "n < 0");
    if (!out || !xs || !ys) return fail(RBS_EINVAL, "null pointer");
    for (int j = 0; j < k; j++)
        if (n > 0 && (!xs[j] || !ys[j])) return fail(RBS_EINVAL, "null operand");
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    const bool out_dev = is_device_ptr(out);
    double *dout = out_dev ? out : w->d_out;
    if (n == 0) {
        if (out_dev) {
            CK(cudaMemsetAsync(out, 0, k * sizeof(double), w->stream));
        } else {
            for (int j = 0; j < k; j++) out[j] = 0.0;
        }
        return RBS_OK;
    }
    const double *dx[KMAX], *dy[KMAX];
    for (int j = 0; j < k; j++) {
        const void *p;
        if ((rc = to_device(w, 2 * j % 8, xs[j], (size_t)n * 8, &p))) return rc;
        dx[j] = (const double *)p;
        if ((rc = to_device(w, (2 * j + 1) % 8, ys[j], (size_t)n * 8, &p))) return rc;
        dy[j] = (const double *)p;
    }
    CK(launch_exdot(k, dx, dy, n, w->g, dout, window_param(), exdot_cfg(w, n, k, window_param()), w->stream));
    if (!out_dev) {
        CK(cudaMemcpyAsync(w->h_out, w->d_out, k * sizeof(double), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        for (int j = 0; j < k; j++) out[j] = w->h_out[j];
    }
    return RBS_OK;
}

int rbs_exdot(const double *x, const double *y, int64_t n, double *out, void *stream) {
    const double *xs[1] = {x}, *ys[1] = {y};
    return exdot_common(1, xs, ys, n, out, stream);
}

int rbs_exdot_multi(int k, const double *const *xs, const double *const *ys, int64_t n, double *out,
                    void *stream) {
    if (k >= 1 && k <= KMAX && xs && ys)
        for (int j = 0; j < k; j++)
            if (n > 0 && (!is_device_ptr(xs[j]) || !is_device_ptr(ys[j])))
                return fail(RBS_EINVAL, "rbs_exdot_multi operands must be device pointers");
    return exdot_common(k, xs, ys, n, out, stream);
}

int rbs_exdot_partial(const double *x, const double *y, int64_t n, int64_t *limbs, int32_t *flags,
                      void *stream) {
    if (n < 0 || !limbs || !flags || (n > 0 && (!x || !y))) return fail(RBS_EINVAL, "bad argument");
    if (!is_device_ptr(limbs) || !is_device_ptr(flags) || (n > 0 && (!is_device_ptr(x) || !is_device_ptr(y))))
        return fail(RBS_EINVAL, "rbs_exdot_partial takes device pointers");
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    if (n == 0) {
        CK(cudaMemsetAsync(limbs, 0, RBS_LIMBS * sizeof(int64_t), w->stream));
        CK(cudaMemsetAsync(flags, 0, sizeof(int32_t), w->stream));
        return RBS_OK;
    }
    CK(launch_exdot_partial(x, y, n, w->g, limbs, flags, 4, exdot_cfg(w, n, 1, 4), w->stream));
    return RBS_OK;
}

int rbs_round_limbs(const int64_t *limbs, const int32_t *flags, double *out, void *stream) {
    if (!limbs || !flags || !out) return fail(RBS_EINVAL, "null pointer");
    if (!is_device_ptr(limbs) || !is_device_ptr(flags)) return fail(RBS_EINVAL, "limbs/flags must be device pointers");
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    const bool out_dev = is_device_ptr(out);
    CK(launch_round_limbs(limbs, flags, out_dev ? out : w->d_out, w->stream));
    if (!out_dev) {
        CK(cudaMemcpyAsync(w->h_out, w->d_out, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        *out = w->h_out[0];
    }
    return RBS_OK;
}

static int check_csr_args(const rbs_csr *A) {
    if (!A) return fail(RBS_EINVAL, "A is null");
    if (A->n <= 0 || A->n > 0x7fffffff) return fail(RBS_EINVAL, "A->n must be in 1..2^31-1");
    if (A->nnz < 0) return fail(RBS_EINVAL, "A->nnz < 0");
    if (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val))) return fail(RBS_EINVAL, "null CSR array");
    return RBS_OK;
}

int rbs_spmv_csr(const rbs_csr *A, const double *x, double *y, void *stream) {
    int rc = check_csr_args(A);
    if (rc) return rc;
    if (!x || !y) return fail(RBS_EINVAL, "null vector");
    if (x == y) return fail(RBS_EINVAL, "y must not alias x");
    Workspace *w;
    if ((rc = ws_get((cudaStream_t)stream, &w))) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    CSRArgs a{A->n, A->nnz, A->rowptr, A->col, A->val};
    const int sb = block_of(p_spmv_block.load(), 256);
    const int carve = carveout_param();
    const int mode = spmv_mode_for(A->n, A->nnz);
    Cfg c = grid_for(w, A->n, sb, spmv_blocks_per_sm(sb, carve, mode & SPMV_MODE_MASK));
    c.mode = mode;
    c.carveout = carve;
    CK(launch_spmv(a, x, y, nullptr, &w->g->err, c, w->stream));
    return RBS_OK;
}

int rbs_jacobi_invd(const rbs_csr *A, const double *diag, double *invd, void *stream) {
    int rc = check_csr_args(A);
    if (rc) return rc;
    if (!invd) return fail(RBS_EINVAL, "null invd");
    Workspace *w;
    if ((rc = ws_get((cudaStream_t)stream, &w))) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    CSRArgs a{A->n, A->nnz, A->rowptr, A->col, A->val};
    Cfg c = grid_for(w, A->n, 256, 8);
    CK(launch_jacobi_invd(a, diag, invd, &w->g->err, c, w->stream));
    unsigned err = 0;
    if ((rc = read_err(w, &err))) return rc;
    if (err & 2u) return fail(RBS_EINVAL, "zero, NaN or missing diagonal entry");
    if (err) return fail(RBS_EINVAL, "invalid CSR row pointers");
    return RBS_OK;
}

int rbs_jacobi_apply(int64_t n, const double *invd, const double *p, double *phat, void *stream) {
    if (n < 0 || (n > 0 && (!invd || !p || !phat))) return fail(RBS_EINVAL, "bad argument");
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    if (n == 0) return RBS_OK;
    CK(launch_jacobi_apply(n, invd, p, phat, grid_for(w, n, 256, 8), w->stream));
    return RBS_OK;
}

int rbs_solve(const rbs_csr *A, const double *b, const double *x0, const double *jacobi_diag, double tol,
              int32_t maxit, int32_t variant, double *x_out, rbs_info *info, rbs_history *hist,
              void *stream) {
    return rbs_solve_ex(A, b, x0, jacobi_diag, tol, maxit, variant, nullptr, x_out, info, hist, nullptr,
                        stream);
}

int rbs_solve_ex(const rbs_csr *A, const double *b, const double *x0, const double *jacobi_diag,
                 double tol, int32_t maxit, int32_t variant, const rbs_opts *opts, double *x_out,
                 rbs_info *info, rbs_history *hist, rbs_prof *prof, void *stream) {
    if (info) memset(info, 0, sizeof *info);
    if (info) info->status = RBS_EINVAL;
    int rc = check_csr_args(A);
    if (rc) return rc;
    if (!b || !x_out || !info) return fail(RBS_EINVAL, "null b, x_out or info");
    if (maxit < 0 || !(tol >= 0.0)) return fail(RBS_EINVAL, "maxit < 0 or tol not >= 0");
    if (variant != RBS_CLASSIC && variant != RBS_PIPELINED) return fail(RBS_EINVAL, "unknown variant");
    if (hist && (hist->cap < 0 || (hist->cap > 0 && !hist->rec))) return fail(RBS_EINVAL, "bad history");
    rbs_opts o{};
    if (opts) o = *opts;
    if (o.dot_mode != RBS_DOT_EXACT && o.dot_mode != RBS_DOT_PLAIN) return fail(RBS_EINVAL, "bad dot_mode");
    if (o.loop_mode != RBS_LOOP_GRAPH && o.loop_mode != RBS_LOOP_HOST) return fail(RBS_EINVAL, "bad loop_mode");
    if (prof) {
        // keep the caller's trace buffers, clear the counters
        rbs_prof keep = *prof;
        memset(prof, 0, sizeof *prof);
        prof->trace_cap = keep.trace_cap;
        prof->trace_kind = keep.trace_kind;
        prof->trace_iter = keep.trace_iter;
        prof->trace_ms = keep.trace_ms;
    }

    Workspace *w;
    if ((rc = ws_get((cudaStream_t)stream, &w))) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    const int64_t n = A->n, nnz = A->nnz;

    // caller buffers, staged to the device when they live in host memory
    const void *rowptr, *col, *val, *db, *dx0 = nullptr, *ddiag = nullptr;
    if ((rc = to_device(w, 0, A->rowptr, (size_t)(n + 1) * 8, &rowptr))) return rc;
    if ((rc = to_device(w, 1, A->col, (size_t)nnz * 4, &col))) return rc;
    if ((rc = to_device(w, 2, A->val, (size_t)nnz * 8, &val))) return rc;
    if ((rc = to_device(w, 3, b, (size_t)n * 8, &db))) return rc;
    if (x0 && (rc = to_device(w, 4, x0, (size_t)n * 8, &dx0))) return rc;
    if (jacobi_diag && (rc = to_device(w, 5, jacobi_diag, (size_t)n * 8, &ddiag))) return rc;

    // solver vectors, 256-byte aligned each
    const size_t stride = ((size_t)n * 8 + 255) / 256 * 256;
    CK(ensure(w->vec, stride * NVEC));
    double *vp[NVEC];
    for (int i = 0; i < NVEC; i++) vp[i] = (double *)((char *)w->vec.p + stride * i);
    const bool xout_dev = is_device_ptr(x_out) && ((uintptr_t)x_out % 16 == 0);
    SolverVecs V;
    V.x = xout_dev ? x_out : vp[0];
    V.r = vp[1]; V.r0 = vp[2]; V.p = vp[3]; V.ph = vp[4]; V.s = vp[5]; V.q = vp[6]; V.qh = vp[7];
    V.y = vp[8]; V.invd = vp[9]; V.rh = vp[10]; V.w = vp[11]; V.wh = vp[12]; V.t = vp[13];
    V.sh = vp[14]; V.z = vp[15]; V.zh = vp[16]; V.v = vp[17];

    const int hcap = hist ? (hist->cap < maxit ? hist->cap : maxit) : 0;
    CK(ensure(w->hist, (size_t)(hcap > 0 ? hcap : 1) * RBS_HIST_W * 8));

    SolverState *h = w->h_st;
    memset(h, 0, sizeof *h);
    h->tol = tol;
    h->maxit = maxit;
    h->variant = variant;
    h->hist_cap = hcap;
    CK(cudaMemcpyAsync(w->st, h, sizeof *h, cudaMemcpyHostToDevice, w->stream));
    CK(cudaMemsetAsync(&w->g->err, 0, sizeof(unsigned), w->stream));

    SolverArgs a;
    memset(&a, 0, sizeof a);  // padding too: the struct keys the graph cache
    a.A = CSRArgs{n, nnz, (const int64_t *)rowptr, (const int32_t *)col, (const double *)val};
    a.v = V;
    a.b = (const double *)db;
    a.x0 = (const double *)dx0;
    a.st = w->st;
    a.g = w->g;
    a.hist = (double *)w->hist.p;
    a.err = &w->g->err;
    a.dot_mode = o.dot_mode;
    {
        const int vb = block_of(p_vec_block.load(), 256);
        const int carve = carveout_param();
        const int smode = spmv_mode_for(n, nnz);
        const int bps = solver_blocks_per_sm(variant, o.dot_mode, 1, vb, carve, smode & SPMV_MODE_MASK);
        a.vec = grid_for(w, (n + 1) / 2, vb, bps);
        a.p3 = variant == RBS_PIPELINED
                   ? grid_for(w, (n + 1) / 2, vb, solver_blocks_per_sm(variant, o.dot_mode, 2, vb, carve,
                                                                       smode & SPMV_MODE_MASK))
                   : a.vec;
        if (p_vec_grid.load() > 0) a.vec.grid = a.p3.grid = (int)p_vec_grid.load();
        // long rows: the register-staged kernels' own block (the knob is for short rows)
        const int sb = (smode & SPMV_MODE_MASK) == SPMV_MODE_LONG ? SPMV_REG_WARPS * 32
                                                                  : block_of(p_spmv_block.load(), 256);
        a.spmv = grid_for(w, n, sb, solver_blocks_per_sm(variant, o.dot_mode, 0, sb, carve, smode & SPMV_MODE_MASK));
        a.spmv.mode = smode;
        a.k3 = variant == RBS_CLASSIC
                   ? grid_for(w, n, sb, solver_blocks_per_sm(variant, o.dot_mode, 3, sb, carve, smode & SPMV_MODE_MASK))
                   : a.spmv;
        a.k3.mode = smode;
        a.carveout = carveout_param();
        a.spmv.carveout = a.carveout;
        a.k3.carveout = a.carveout;
        // window headroom: at most 2^20 products per thread per launch
        const int64_t minv = (n + ((int64_t)a.vec.block << 20) - 1) / ((int64_t)a.vec.block << 20);
        if (a.vec.grid < minv) a.vec.grid = (int)minv;
        if (a.p3.grid < minv) a.p3.grid = (int)minv;
        const int64_t mins = (n + ((int64_t)a.spmv.block << 20) - 1) / ((int64_t)a.spmv.block << 20);
        if (a.spmv.grid < mins) a.spmv.grid = (int)mins;
        if (a.k3.grid < mins) a.k3.grid = (int)mins;
    }

    // structure check and Jacobi set-up (Sec. 4: M = diag(A))
    CK(launch_csr_check(a.A, &w->g->err, grid_for(w, nnz > n ? nnz : n, 256, 8), w->stream));
    CK(launch_jacobi_invd(a.A, (const double *)ddiag, V.invd, &w->g->err, grid_for(w, n, 256, 8), w->stream));
    unsigned err = 0;
    if ((rc = read_err(w, &err))) return rc;
    if (err & 1u) return fail(RBS_EINVAL, "invalid CSR structure");
    if (err & 2u) return fail(RBS_EINVAL, "zero, NaN or missing diagonal entry");

    EventTimer timer(w);
    KernelTimer *tm = (o.profile && prof) ? &timer : nullptr;
    CK(solver_setup(a, variant, w->stream, tm));

    const bool use_graph = !tm && o.loop_mode == RBS_LOOP_GRAPH && maxit > 0;
    if (use_graph) {
        if ((rc = graph_loop(w, a, variant))) return rc;
    }
    int chunk = o.check_every > 0 ? o.check_every : (p_check_every.load() > 0 ? (int)p_check_every.load() : 8);
    if (!use_graph && w->ev_chunk.size() < 2) {
        for (int i = (int)w->ev_chunk.size(); i < 2; i++) {
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            w->ev_chunk.push_back(e);
        }
    }
    // keep one chunk of iterations enqueued ahead of the flag being read
    int64_t launched = 0;
    int slot = 0, prev = -1;
    while (!use_graph) {
        int cur = -1;
        if (launched < maxit) {
            int m = (int)((maxit - launched) < chunk ? (maxit - launched) : chunk);
            for (int i = 0; i < m; i++) {
                if (tm) timer.begin_iteration((int)(launched + i));
                CK(solver_iteration(a, variant, w->stream, tm));
            }
            launched += m;
            cur = slot;
            CK(cudaMemcpyAsync(&w->h_flags[cur], &w->st->done, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               w->stream));
            CK(cudaEventRecord(w->ev_chunk[cur], w->stream));
            if (tm) tm->gap();
            slot ^= 1;
        }
        if (prev >= 0) {
            CK(cudaEventSynchronize(w->ev_chunk[prev]));
            if (w->h_flags[prev]) break;
        }
        if (cur < 0) break;
        prev = cur;
    }
    CK(cudaMemcpyAsync(h, w->st, sizeof *h, cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    if ((rc = read_err(w, &err))) return rc;
    if (err & 4u) return fail(RBS_ETIMEOUT, "a bounded wait on an asynchronous copy expired");
    if (err) return fail(RBS_EINVAL, "a kernel met an out-of-range CSR index");

    info->iters = h->iter;
    info->status = h->status;
    info->tau0 = h->tau0;
    info->tau_final = h->tau;
    info->rho0 = h->rho0;
    info->tau_max = h->tau_max;
    info->alpha0 = variant == RBS_PIPELINED ? h->alpha0 : __builtin_nan("");
    info->mu0 = variant == RBS_PIPELINED ? h->mu0 : 0.0;
    info->converged = (h->status == RBS_OK && !(h->tau > h->tau_max)) ? 1 : 0;
    if (hist) {
        hist->len = h->iter < hcap ? h->iter : hcap;
        if (hist->len > 0)
            CK(cudaMemcpyAsync(hist->rec, w->hist.p, (size_t)hist->len * RBS_HIST_W * 8,
                               cudaMemcpyDeviceToHost, w->stream));
    }
    if (!xout_dev)
        CK(cudaMemcpyAsync(x_out, V.x, (size_t)n * 8,
                           is_device_ptr(x_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    if (tm) {
        // launches that returned at once on the stop flag are traced but not
        // counted: every launch of an iteration index >= iters, and in the last
        // iteration those after the stopping kernel (classic K5, pipelined S18)
        const int last_slot = variant == RBS_CLASSIC ? 4 : 3;
        const bool trace = prof->trace_cap > 0 && prof->trace_kind && prof->trace_iter && prof->trace_ms;
        for (auto &r : timer.rec) {
            if (!r.b) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
            if (trace && prof->trace_len < prof->trace_cap) {
                prof->trace_kind[prof->trace_len] = r.kind;
                prof->trace_iter[prof->trace_len] = r.iter;
                prof->trace_ms[prof->trace_len] = ms;
                prof->trace_len++;
            }
            const bool ran = r.iter < h->iter && !(r.iter == h->iter - 1 && r.slot == last_slot && h->done);
            if (ran && r.kind >= 0 && r.kind < RBS_PROF_KINDS) {
                prof->ms[r.kind] += ms;
                prof->launches[r.kind] += 1;
            }
        }
    }
    if (h->status != RBS_OK)
        return fail(h->status, h->status == RBS_EBREAKDOWN ? "breakdown: zero denominator"
                                                           : "non-finite scalar");
    return RBS_OK;
}

}  // extern "C"

// ---- batched solves and their schedule tuner ---------------------------------

namespace {

std::mutex g_tuned_mu;
std::map<int, rbs_batch_schedule> g_tuned;  // per device: the last tuned schedule

rbs_batch_schedule default_schedule() {
    rbs_batch_schedule d;
    memset(&d, 0, sizeof d);
    d.cluster = 8;
    d.split = 0;  // every system solved by a whole cluster
    return d;
}

bool schedule_ok(const rbs_batch_schedule &s) {
    return s.cluster >= 0 && s.cluster <= 16 && (s.cluster & (s.cluster - 1)) == 0 && s.split >= 0;
}

// The stepped schedule (cluster 0): every system of the batch advances one
// iteration per step, one launch per phase for all of them (the serving
// engine's per-step kernels), each on blocks of `split` rows (0: 8192), so a
// large system runs on as many SMs as its rows fill. The host enqueues steps in
// chunks no longer than any system's remaining iterations (a system runs
// exactly min(maxit, its own stop) iterations), reads every state after each
// chunk and drops the stopped systems from the next chunk's task lists.
// proxy_maxit / ms: as batch_solve.
int batch_stepped(Workspace *w, int32_t nsys, const rbs_system *systems, rbs_info *infos, rbs_history *hists,
                  const rbs_batch_schedule &sched, const int32_t *proxy_maxit, float *ms) {
    const bool proxy = proxy_maxit != nullptr;
    // rows per block: fixed (split > 0), or chosen per chunk from the rows still
    // iterating so that a launch has about four waves of 256-thread blocks --
    // large blocks while the whole batch iterates (each block's flush and
    // cross-block reduction is a fixed cost), small ones once few systems are
    // left (so that they still spread over every SM)
    const int64_t fixed_rows = sched.split > 0 ? (sched.split + 63) / 64 * 64 : 0;
    int64_t rows = fixed_rows ? fixed_rows : 8192;
    auto pick_rows = [&](int64_t active_rows) {
        if (fixed_rows) return fixed_rows;
        const int64_t waves = 4LL * w->sms * 3;
        int64_t r = (active_rows + waves - 1) / waves;
        r = std::max<int64_t>(1024, std::min<int64_t>(65536, r));
        return (r + 63) / 64 * 64;
    };
    std::vector<char> valid((size_t)nsys, 1);
    std::vector<int32_t> maxit((size_t)nsys, 0);
    size_t work_elems = 0, hist_recs = 0;
    for (int i = 0; i < nsys; i++) {
        const rbs_system &S = systems[i];
        memset(&infos[i], 0, sizeof infos[i]);
        bool ok = S.A.n > 0 && S.A.n <= 0x7fffffff && S.A.nnz >= 0 && S.A.rowptr &&
                  (S.A.nnz == 0 || (S.A.col && S.A.val)) && S.b && (S.x || proxy) && S.maxit >= 0 &&
                  S.tol >= 0.0 && (S.variant == RBS_CLASSIC || S.variant == RBS_PIPELINED);
        ok = ok && is_device_ptr(S.A.rowptr) && is_device_ptr(S.b) && (proxy || is_device_ptr(S.x)) &&
             (proxy || ((uintptr_t)S.x & 15) == 0) &&
             (S.A.nnz == 0 || (is_device_ptr(S.A.col) && is_device_ptr(S.A.val))) &&
             (!S.x0 || is_device_ptr(S.x0)) && (!S.jacobi_diag || is_device_ptr(S.jacobi_diag));
        if (hists && (hists[i].cap < 0 || (hists[i].cap > 0 && !hists[i].rec))) ok = false;
        valid[(size_t)i] = ok;
        if (!ok) continue;
        maxit[(size_t)i] = proxy ? std::min(S.maxit, std::max(proxy_maxit[i], 1)) : S.maxit;
        const int64_t stride = (S.A.n + 31) / 32 * 32;
        work_elems += (size_t)stride * ((S.variant == RBS_PIPELINED ? 16 : 9) + (proxy ? 1 : 0));
        const int cap = hists ? std::min(hists[i].cap, S.maxit) : 0;
        hist_recs += (size_t)(cap > 0 ? cap : 0);
    }
    const size_t cb = step_ctx_bytes();
    CK(ensure(w->batch_work, work_elems * 8));
    CK(ensure(w->batch_hist, (hist_recs > 0 ? hist_recs : 1) * RBS_HIST_W * 8));
    CK(ensure(w->step_ctx, (size_t)nsys * cb));
    CK(ensure(w->step_state, (size_t)nsys * sizeof(SolverState)));
    CK(ensure(w->step_scr, (size_t)nsys * sizeof(DotScratch)));
    std::vector<char> hctx((size_t)nsys * cb, 0);
    std::vector<SolverState> hst((size_t)nsys);
    std::vector<double *> hist_dev((size_t)nsys, nullptr);
    std::vector<int32_t> hist_cap((size_t)nsys, 0);
    SolverState *dst = (SolverState *)w->step_state.p;
    DotScratch *dscr = (DotScratch *)w->step_scr.p;
    size_t woff = 0, hoff = 0;
    for (int i = 0; i < nsys; i++) {
        SolverState &h = hst[(size_t)i];
        memset(&h, 0, sizeof h);
        if (!valid[(size_t)i]) {
            h.done = 1;
            h.status = RBS_EINVAL;
            continue;
        }
        const rbs_system &S = systems[i];
        const int64_t stride = (S.A.n + 31) / 32 * 32;
        const int nv = S.variant == RBS_PIPELINED ? 16 : 9;
        double *v[17];
        for (int k = 0; k < nv; k++) v[k] = (double *)w->batch_work.p + woff + (size_t)k * stride;
        woff += (size_t)stride * nv;
        SolverVecs V;
        memset(&V, 0, sizeof V);
        V.x = S.x;
        if (proxy) {
            V.x = (double *)w->batch_work.p + woff;
            woff += (size_t)stride;
        }
        V.r = v[0]; V.r0 = v[1]; V.ph = v[2]; V.s = v[3]; V.q = v[4]; V.qh = v[5]; V.y = v[6]; V.invd = v[7];
        if (S.variant == RBS_CLASSIC) {
            V.p = v[8];
        } else {
            V.rh = v[8]; V.w = v[9]; V.wh = v[10]; V.t = v[11]; V.sh = v[12]; V.z = v[13]; V.zh = v[14]; V.v = v[15];
        }
        const int cap = hists ? std::min(hists[i].cap, S.maxit) : 0;
        hist_cap[(size_t)i] = cap > 0 ? cap : 0;
        if (hist_cap[(size_t)i]) {
            hist_dev[(size_t)i] = (double *)w->batch_hist.p + hoff * RBS_HIST_W;
            hoff += (size_t)hist_cap[(size_t)i];
        }
        h.tol = S.tol;
        h.maxit = maxit[(size_t)i];
        h.variant = S.variant;
        h.hist_cap = hist_cap[(size_t)i];
        CSRArgs A{S.A.n, S.A.nnz, S.A.rowptr, S.A.col, S.A.val};
        step_ctx_make(hctx.data() + (size_t)i * cb, A, V, S.b, S.x0, S.jacobi_diag, dst + i, dscr + i,
                      hist_dev[(size_t)i]);
    }
    // tasks of a set of systems of one variant, appended to `out`
    auto tasks_of = [&](const std::vector<int> &ids, std::vector<StepTask> &out) {
        for (int i : ids) {
            const int64_t n = systems[i].A.n;
            const int nb = (int)((n + rows - 1) / rows);
            for (int b = 0; b < nb; b++)
                out.push_back(StepTask{i, nb, (int64_t)b * rows, std::min(n, (int64_t)(b + 1) * rows)});
        }
    };
    std::vector<int> cls, pipe;
    int64_t all_rows = 0;
    for (int i = 0; i < nsys; i++)
        if (valid[(size_t)i]) {
            (systems[i].variant == RBS_PIPELINED ? pipe : cls).push_back(i);
            all_rows += systems[i].A.n;
        }
    rows = pick_rows(all_rows);
    std::vector<StepTask> tasks;
    tasks_of(cls, tasks);
    const size_t ncls = tasks.size();
    tasks_of(pipe, tasks);
    CK(ensure(w->step_tasks, std::max<size_t>(tasks.size(), 1) * sizeof(StepTask)));
    StepTask *dtask = (StepTask *)w->step_tasks.p;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, w->stream));
    }
    CK(cudaMemcpyAsync(w->step_ctx.p, hctx.data(), (size_t)nsys * cb, cudaMemcpyHostToDevice, w->stream));
    CK(cudaMemcpyAsync(dst, hst.data(), (size_t)nsys * sizeof(SolverState), cudaMemcpyHostToDevice, w->stream));
    CK(cudaMemsetAsync(dscr, 0, (size_t)nsys * sizeof(DotScratch), w->stream));
    if (!tasks.empty())
        CK(cudaMemcpyAsync(dtask, tasks.data(), tasks.size() * sizeof(StepTask), cudaMemcpyHostToDevice, w->stream));
    CK(step_admit(w->step_ctx.p, dtask, (int)ncls, RBS_CLASSIC, w->stream));
    CK(step_admit(w->step_ctx.p, dtask + ncls, (int)(tasks.size() - ncls), RBS_PIPELINED, w->stream));
    CK(cudaMemcpyAsync(hst.data(), dst, (size_t)nsys * sizeof(SolverState), cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    std::vector<int32_t> ran((size_t)nsys, 0);
    auto live = [&](int i) { return !hst[(size_t)i].done && ran[(size_t)i] < maxit[(size_t)i]; };
    // classic and pipelined systems step on two streams (independent work that
    // fills the GPU better once few systems are left), joined after each chunk
    if (!w->side) CK(cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking));
    if (!w->ev_fork) CK(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
    if (!w->ev_join) CK(cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming));
    CK(ensure_host(w->h_states, (size_t)nsys * sizeof(SolverState)));
    SolverState *pst = (SolverState *)w->h_states.p;
    for (;;) {
        std::vector<int> c2, p2;
        int32_t chunk = 8;
        int64_t live_rows = 0;
        for (int i : cls)
            if (live(i)) c2.push_back(i), chunk = std::min(chunk, maxit[(size_t)i] - ran[(size_t)i]),
                         live_rows += systems[i].A.n;
        for (int i : pipe)
            if (live(i)) p2.push_back(i), chunk = std::min(chunk, maxit[(size_t)i] - ran[(size_t)i]),
                         live_rows += systems[i].A.n;
        if (c2.empty() && p2.empty()) break;
        rows = pick_rows(live_rows);
        tasks.clear();
        tasks_of(c2, tasks);
        const size_t nc = tasks.size();
        tasks_of(p2, tasks);
        // the pinned task list is rewritten only after the previous chunk's
        // copy from it has completed (the stream was synchronised)
        CK(ensure_host(w->h_tasks, tasks.size() * sizeof(StepTask)));
        memcpy(w->h_tasks.p, tasks.data(), tasks.size() * sizeof(StepTask));
        CK(cudaMemcpyAsync(dtask, w->h_tasks.p, tasks.size() * sizeof(StepTask), cudaMemcpyHostToDevice, w->stream));
        const int np = (int)(tasks.size() - nc);
        if (np > 0) {
            CK(cudaEventRecord(w->ev_fork, w->stream));
            CK(cudaStreamWaitEvent(w->side, w->ev_fork, 0));
        }
        for (int k = 0; k < chunk; k++) {
            CK(step_iteration(w->step_ctx.p, dtask, (int)nc, RBS_CLASSIC, w->stream));
            CK(step_iteration(w->step_ctx.p, dtask + nc, np, RBS_PIPELINED, w->side));
        }
        if (np > 0) {
            CK(cudaEventRecord(w->ev_join, w->side));
            CK(cudaStreamWaitEvent(w->stream, w->ev_join, 0));
        }
        for (int i : c2) ran[(size_t)i] += chunk;
        for (int i : p2) ran[(size_t)i] += chunk;
        CK(cudaMemcpyAsync(pst, dst, (size_t)nsys * sizeof(SolverState), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        memcpy(hst.data(), pst, (size_t)nsys * sizeof(SolverState));
    }
    if (ms) {
        CK(cudaEventRecord(e1, w->stream));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    int ret = RBS_OK;
    for (int i = 0; i < nsys; i++) {
        rbs_info &I = infos[i];
        const SolverState &q = hst[(size_t)i];
        if (!valid[(size_t)i] || q.status == RBS_EINVAL) {
            I.status = RBS_EINVAL;
            ret = RBS_EINVAL;
            if (hists) hists[i].len = 0;
            continue;
        }
        I.iters = q.iter;
        I.status = q.status;
        I.converged = (q.status == RBS_OK && !(q.tau > q.tau_max)) ? 1 : 0;
        I.tau0 = q.tau0;
        I.tau_final = q.tau;
        I.rho0 = q.rho0;
        I.tau_max = q.tau_max;
        I.alpha0 = systems[i].variant == RBS_PIPELINED ? q.alpha0 : __builtin_nan("");
        I.mu0 = systems[i].variant == RBS_PIPELINED ? q.mu0 : 0.0;
        if (hists) {
            hists[i].len = std::min(q.iter, hist_cap[(size_t)i]);
            if (hists[i].len > 0)
                CK(cudaMemcpy(hists[i].rec, hist_dev[(size_t)i], (size_t)hists[i].len * RBS_HIST_W * 8,
                              cudaMemcpyDeviceToHost));
        }
    }
    if (ret) fail(ret, "one or more systems failed the argument or structure checks");
    return ret;
}

// Solve the batch with schedule `sched`. With proxy_maxit (nsys entries) each
// system stops after that many iterations and writes x into library scratch
// instead of the caller's buffer (the tuner's timing runs); *ms gets the
// device time of the prepare + solve launches.
int batch_solve(Workspace *w, int32_t nsys, const rbs_system *systems, rbs_info *infos, rbs_history *hists,
                const rbs_batch_schedule &sched, const int32_t *proxy_maxit, float *ms) {
    if (sched.cluster == 0) return batch_stepped(w, nsys, systems, infos, hists, sched, proxy_maxit, ms);
    std::vector<BatchSys> sys((size_t)nsys);
    std::vector<char> valid((size_t)nsys, 1);
    size_t work_elems = 0, hist_recs = 0;
    const bool proxy = proxy_maxit != nullptr;
    for (int i = 0; i < nsys; i++) {
        const rbs_system &S = systems[i];
        memset(&infos[i], 0, sizeof infos[i]);
        bool ok = S.A.n > 0 && S.A.n <= 0x7fffffff && S.A.nnz >= 0 && S.A.rowptr &&
                  (S.A.nnz == 0 || (S.A.col && S.A.val)) && S.b && (S.x || proxy) && S.maxit >= 0 &&
                  S.tol >= 0.0 && (S.variant == RBS_CLASSIC || S.variant == RBS_PIPELINED);
        ok = ok && is_device_ptr(S.A.rowptr) && is_device_ptr(S.b) && (proxy || is_device_ptr(S.x)) &&
             (S.A.nnz == 0 || (is_device_ptr(S.A.col) && is_device_ptr(S.A.val))) &&
             (!S.x0 || is_device_ptr(S.x0)) && (!S.jacobi_diag || is_device_ptr(S.jacobi_diag));
        if (hists && (hists[i].cap < 0 || (hists[i].cap > 0 && !hists[i].rec))) ok = false;
        valid[(size_t)i] = ok;
        if (!ok) continue;
        const int64_t stride = (S.A.n + 31) / 32 * 32;
        work_elems += (size_t)stride * ((S.variant == RBS_PIPELINED ? 17 : 9) + (proxy ? 1 : 0));
        const int cap = hists ? std::min(hists[i].cap, S.maxit) : 0;
        hist_recs += (size_t)(cap > 0 ? cap : 0);
    }
    CK(ensure(w->batch_work, work_elems * 8));
    CK(ensure(w->batch_hist, (hist_recs > 0 ? hist_recs : 1) * RBS_HIST_W * 8));
    CK(ensure(w->batch_sys, (size_t)nsys * sizeof(BatchSys)));
    CK(ensure(w->batch_order, ((size_t)nsys * sizeof(int32_t) + 7) / 8 * 8 + (size_t)nsys * sizeof(int64_t)));
    CK(ensure(w->batch_out, (size_t)nsys * sizeof(BatchOut)));
    CK(ensure(w->batch_queue, 16));
    size_t woff = 0, hoff = 0;
    std::vector<int32_t> order;
    for (int i = 0; i < nsys; i++) {
        BatchSys &B = sys[(size_t)i];
        memset(&B, 0, sizeof B);
        if (!valid[(size_t)i]) continue;
        const rbs_system &S = systems[i];
        B.A = CSRArgs{S.A.n, S.A.nnz, S.A.rowptr, S.A.col, S.A.val};
        B.b = S.b;
        B.x0 = S.x0;
        B.diag = S.jacobi_diag;
        B.stride = (S.A.n + 31) / 32 * 32;
        B.work = (double *)w->batch_work.p + woff;
        woff += (size_t)B.stride * (S.variant == RBS_PIPELINED ? 17 : 9);
        if (proxy) {
            B.x = (double *)w->batch_work.p + woff;
            woff += (size_t)B.stride;
        } else {
            B.x = S.x;
        }
        B.tol = S.tol;
        B.maxit = proxy ? std::min(S.maxit, std::max(proxy_maxit[i], 1)) : S.maxit;
        B.variant = S.variant;
        const int cap = hists ? std::min(hists[i].cap, S.maxit) : 0;
        B.hist_cap = cap > 0 ? cap : 0;
        B.hist = B.hist_cap ? (double *)w->batch_hist.p + hoff * RBS_HIST_W : nullptr;
        hoff += (size_t)B.hist_cap;
        order.push_back(i);
    }
    // largest systems first (then by index, so the order is deterministic)
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return systems[a].A.nnz + systems[a].A.n > systems[b].A.nnz + systems[b].A.n;
    });
    const int nq = (int)order.size();
    std::vector<int64_t> sizes((size_t)nq);
    for (int q = 0; q < nq; q++) sizes[(size_t)q] = systems[order[(size_t)q]].A.n;
    int32_t *d_order = (int32_t *)w->batch_order.p;
    int64_t *d_sizes = (int64_t *)((char *)w->batch_order.p + (((size_t)nsys * sizeof(int32_t) + 7) / 8 * 8));
    CK(cudaMemcpyAsync(w->batch_sys.p, sys.data(), (size_t)nsys * sizeof(BatchSys), cudaMemcpyHostToDevice,
                       w->stream));
    if (nq > 0) {
        CK(cudaMemcpyAsync(d_order, order.data(), (size_t)nq * sizeof(int32_t), cudaMemcpyHostToDevice, w->stream));
        CK(cudaMemcpyAsync(d_sizes, sizes.data(), (size_t)nq * sizeof(int64_t), cudaMemcpyHostToDevice, w->stream));
    }
    BatchSchedule b;
    b.cluster = sched.cluster;
    b.split = sched.split;
    b.clusters = 0;
    if (nq > 0) {
        const int fit = batch_max_clusters(b.cluster);
        if (fit < 1) return fail(RBS_EINVAL, "no cluster of this size fits on the device");
        b.clusters = std::max(1, std::min(fit, nq));
    }
    // the batch's device work: zero the outcomes and the queue, check and set
    // up every system (Jacobi), then the persistent solve launch
    auto enqueue = [&](cudaStream_t st) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(w->batch_out.p, 0, (size_t)nsys * sizeof(BatchOut), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w->batch_queue.p, 0, 16, st);
        if (e == cudaSuccess && nq > 0)
            e = launch_batch_prepare((const BatchSys *)w->batch_sys.p, nsys, (BatchOut *)w->batch_out.p, st);
        if (e == cudaSuccess && nq > 0)
            e = launch_batch((const BatchSys *)w->batch_sys.p, d_order, d_sizes, nq, (unsigned *)w->batch_queue.p,
                             (BatchOut *)w->batch_out.p, b, st);
        return e;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the graph is keyed by everything captured launches bake in: descriptors, order,
    // schedule and the workspace buffers they point to
    std::string key;
    if (!ms) {
        key.assign((const char *)sys.data(), sys.size() * sizeof(BatchSys));
        key.append((const char *)order.data(), order.size() * sizeof(int32_t));
        key.append((const char *)&b, sizeof b);
        const void *bufs[] = {w->batch_sys.p, w->batch_order.p, w->batch_out.p, w->batch_queue.p};
        key.append((const char *)bufs, sizeof bufs);
    }
    const bool replay = !ms && w->batch_exec && key == w->batch_key;
    const bool capture = !ms && !replay && key == w->batch_seen;
    if (!replay && !capture) {
        // tuner trials (timed) and a batch seen for the first time: plain launches
        if (ms) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, w->stream));
        } else {
            w->batch_seen = key;
        }
        CK(enqueue(w->stream));
    } else {
        // a repeated system set and schedule: one graph, captured once, replayed
        if (capture) {
            std::lock_guard<std::mutex> cap(g_cap_mu);
            if (w->batch_exec) cudaGraphExecDestroy(w->batch_exec);
            w->batch_exec = nullptr;
            w->batch_key.clear();
            if (!w->cap) CK(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e1c = enqueue(w->cap);
            cudaGraph_t gr = nullptr;
            const cudaError_t e2c = cudaStreamEndCapture(w->cap, &gr);
            if (e1c != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                return cuda_fail(e1c, "capture of the batched solve");
            }
            if (e2c != cudaSuccess) return cuda_fail(e2c, "cudaStreamEndCapture (batched solve)");
            cudaGraphExec_t ex = nullptr;
            const cudaError_t e3c = cudaGraphInstantiate(&ex, gr, 0);
            cudaGraphDestroy(gr);
            if (e3c != cudaSuccess) return cuda_fail(e3c, "cudaGraphInstantiate (batched solve)");
            w->batch_exec = ex;
            w->batch_key = key;
            w->batch_seen.clear();
        }
        CK(cudaGraphLaunch(w->batch_exec, w->stream));
    }
    if (ms) {
        CK(cudaEventRecord(e1, w->stream));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    std::vector<BatchOut> out((size_t)nsys);
    CK(cudaMemcpyAsync(out.data(), w->batch_out.p, (size_t)nsys * sizeof(BatchOut), cudaMemcpyDeviceToHost,
                       w->stream));
    CK(cudaStreamSynchronize(w->stream));
    int ret = RBS_OK;
    for (int i = 0; i < nsys; i++) {
        rbs_info &I = infos[i];
        const BatchOut &O = out[(size_t)i];
        if (!valid[(size_t)i] || O.err) {
            I.status = RBS_EINVAL;
            ret = RBS_EINVAL;
            if (hists) hists[i].len = 0;
            continue;
        }
        I.iters = O.iters;
        I.converged = O.converged;
        I.status = O.status;
        I.tau0 = O.tau0;
        I.tau_final = O.tau_final;
        I.rho0 = O.rho0;
        I.tau_max = O.tau_max;
        I.alpha0 = systems[i].variant == RBS_PIPELINED ? O.alpha0 : __builtin_nan("");
        I.mu0 = systems[i].variant == RBS_PIPELINED ? O.mu0 : 0.0;
        if (hists) {
            const BatchSys &B = sys[(size_t)i];
            hists[i].len = std::min(O.iters, B.hist_cap);
            if (hists[i].len > 0)
                CK(cudaMemcpy(hists[i].rec, B.hist, (size_t)hists[i].len * RBS_HIST_W * 8, cudaMemcpyDeviceToHost));
        }
    }
    if (ret) fail(ret, "one or more systems failed the argument or structure checks");
    return ret;
}

}  // namespace

extern "C" int rbs_solve_batched_ex(int32_t nsys, const rbs_system *systems, rbs_info *infos, rbs_history *hists,
                                    const rbs_batch_schedule *sched, void *stream) {
    if (nsys < 0 || (nsys > 0 && (!systems || !infos))) return fail(RBS_EINVAL, "bad batch arguments");
    if (sched && !schedule_ok(*sched)) return fail(RBS_EINVAL, "bad batch schedule");
    if (nsys == 0) return RBS_OK;
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    rbs_batch_schedule use = default_schedule();
    if (sched) {
        use = *sched;
    } else {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(w->dev);
        if (it != g_tuned.end()) use = it->second;
    }
    std::lock_guard<std::mutex> lk(w->mu);
    return batch_solve(w, nsys, systems, infos, hists, use, nullptr, nullptr);
}

extern "C" int rbs_solve_batched(int32_t nsys, const rbs_system *systems, rbs_info *infos, rbs_history *hists,
                                 void *stream) {
    return rbs_solve_batched_ex(nsys, systems, infos, hists, nullptr, stream);
}

extern "C" int rbs_batch_tune(int32_t nsys, const rbs_system *systems, const rbs_info *prev, int32_t proxy_iters,
                              rbs_batch_schedule *best, void *stream) {
    if (nsys < 1 || !systems || !best || proxy_iters < 1) return fail(RBS_EINVAL, "bad tuning arguments");
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(w->mu);
    // proxy iteration caps: a fixed number, or a fraction of a previous solve's
    // counts so that the systems keep their relative costs
    std::vector<int32_t> cap((size_t)nsys, proxy_iters);
    if (prev) {
        int32_t mx = 1;
        for (int i = 0; i < nsys; i++) mx = std::max(mx, prev[i].iters);
        for (int i = 0; i < nsys; i++)
            cap[(size_t)i] = std::max(1, (int32_t)((int64_t)prev[i].iters * proxy_iters / mx));
    }
    // split candidates: quantiles of the system sizes
    std::vector<int64_t> n;
    for (int i = 0; i < nsys; i++) n.push_back(systems[i].A.n);
    std::sort(n.begin(), n.end());
    auto quant = [&](double f) { return n[(size_t)std::min<double>((double)n.size() - 1, f * (double)n.size())]; };
    std::vector<int64_t> splits = {0, quant(0.5), quant(0.75), quant(0.9), n.back() + 1};
    std::vector<rbs_info> infos((size_t)nsys);
    rbs_batch_schedule top = default_schedule();
    float top_ms = -1.f;
    auto trial = [&](int cluster, int64_t split) -> int {
        rbs_batch_schedule s = default_schedule();
        s.cluster = cluster;
        s.split = split;
        if (cluster > 0 && batch_max_clusters(cluster) < 1) return RBS_OK;
        float ms = 0.f;
        int r = batch_solve(w, nsys, systems, infos.data(), nullptr, s, cap.data(), &ms);
        if (r && r != RBS_EINVAL) return r;
        if (top_ms < 0.f || ms < top_ms) {
            top = s;
            top_ms = ms;
        }
        return RBS_OK;
    };
    // cluster sizes at the median split, then every split for the best size
    for (int c : {1, 2, 4, 8, 16})
        if ((rc = trial(c, c == 1 ? 0 : splits[1]))) return rc;
    const int bestc = top.cluster;
    if (bestc > 1)
        for (size_t k = 0; k < splits.size(); k++)
            if (k != 1 && (rc = trial(bestc, splits[k]))) return rc;
    // the stepped schedule (cluster 0): adaptive block size, then two fixed ones
    for (int64_t rows : {0, 2048, 8192})
        if ((rc = trial(0, rows))) return rc;
    top.ms = top_ms;
    *best = top;
    std::lock_guard<std::mutex> lk2(g_tuned_mu);
    g_tuned[w->dev] = top;
    return RBS_OK;
}

extern "C" int rbs_fpe_dot(const double *x, const double *y, int64_t n, double *out, int32_t *fell_back,
                           void *stream) {
    if (n < 0 || !out || (n > 0 && (!x || !y))) return fail(RBS_EINVAL, "bad argument");
    if (fell_back) *fell_back = 0;
    Workspace *w;
    int rc = ws_get((cudaStream_t)stream, &w);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(w->mu);
        if (n == 0) {
            if (is_device_ptr(out)) CK(cudaMemsetAsync(out, 0, sizeof(double), w->stream));
            else *out = 0.0;
            return RBS_OK;
        }
        const void *dx, *dy;
        if ((rc = to_device(w, 0, x, (size_t)n * 8, &dx))) return rc;
        if ((rc = to_device(w, 1, y, (size_t)n * 8, &dy))) return rc;
        CK(cudaMemsetAsync(&w->g->err, 0, sizeof(unsigned), w->stream));
        const int fb = block_of(p_exdot_block.load(), 256);
        Cfg c = persistent_cfg(w, n, fpe_blocks_per_sm(fb), fb);
        CK(launch_fpe_dot((const double *)dx, (const double *)dy, n, w->g, w->d_out, &w->g->err, c, w->stream));
        unsigned lost = 0;
        if ((rc = read_err(w, &lost))) return rc;
        if (!lost) {
            if (is_device_ptr(out)) {
                CK(cudaMemcpyAsync(out, w->d_out, sizeof(double), cudaMemcpyDeviceToDevice, w->stream));
            } else {
                CK(cudaMemcpyAsync(w->h_out, w->d_out, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
                CK(cudaStreamSynchronize(w->stream));
                *out = w->h_out[0];
            }
            return RBS_OK;
        }
    }
    // the expansions could not hold every bit: the exact dot instead
    if (fell_back) *fell_back = 1;
    return rbs_exdot(x, y, n, out, stream);
}
