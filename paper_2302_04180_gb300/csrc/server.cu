// Serving runtime: a request loop with per-iteration continuous batching.
//
// Clients submit solves (rbs_system, device data) at any time. An engine
// thread owns a CUDA stream and a set of slots, each the resident state of one
// system in flight (its Krylov vectors, device scalars and dot scratch). The
// engine advances in steps: a step admits pending requests into free slots
// while their vector memory fits the budget (their structure check, Jacobi
// set-up and solver set-up run in that step), then runs one iteration of every
// system in flight -- one launch per phase for all of them (kernels_step.cu),
// each system on blocks in proportion to its rows -- and copies every slot's
// device scalars back. Steps are pipelined: the engine reads a step's scalars
// a step or two later, retires the systems that have stopped (or reached
// maxit), frees their memory in stream order and lets their slots be reused
// once no enqueued step refers to them. A request that arrives while others
// iterate joins them at the next step. Each answer is bitwise the one rbs_solve
// gives for that system alone (same element functions, same dot reductions,
// same scalar tails). Latency is measured from submission to retirement.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.h"
#include "rbs.h"

namespace rbs {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    rbs_system sys;
    int64_t bytes;  // device memory of its Krylov vectors while in flight
    Clock::time_point submitted, started, finished;
    rbs_info info;
    bool done;
    int64_t admit_step, finish_step;
    int32_t active_at_admit;  // systems already in flight on its engine when it joined
    std::string error;        // message of a request that failed as a whole
};

int nvec_of(int variant) { return variant == RBS_PIPELINED ? 16 : 9; }
int64_t stride_of(int64_t n) { return (n + 31) / 32 * 32; }  // 256-byte aligned vectors
int64_t state_bytes(const rbs_system &s) { return stride_of(s.A.n) * 8 * nvec_of(s.variant); }

bool dev_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Argument checks done at submission (the structure checks run on the device).
const char *bad_system(const rbs_system &s) {
    if (s.A.n <= 0 || s.A.n > 0x7fffffff || s.A.nnz < 0) return "bad matrix size";
    if (!s.A.rowptr || (s.A.nnz > 0 && (!s.A.col || !s.A.val)) || !s.b || !s.x) return "null pointer";
    if (s.maxit < 0 || !(s.tol >= 0.0)) return "maxit < 0 or tol not >= 0";
    if (s.variant != RBS_CLASSIC && s.variant != RBS_PIPELINED) return "unknown variant";
    if (((uintptr_t)s.x & 15) != 0) return "x must be 16-byte aligned";
    if (!dev_ptr(s.A.rowptr) || !dev_ptr(s.b) || !dev_ptr(s.x) ||
        (s.A.nnz > 0 && (!dev_ptr(s.A.col) || !dev_ptr(s.A.val))) || (s.x0 && !dev_ptr(s.x0)) ||
        (s.jacobi_diag && !dev_ptr(s.jacobi_diag)))
        return "the server takes device pointers";
    return nullptr;
}

constexpr int RING = 8;   // steps whose task lists and scalar copies may be in flight
constexpr int DEPTH = 2;  // steps enqueued ahead of the last one read back

}  // namespace

struct Server {
    int device = 0;
    int slots = 64;
    int64_t seg_rows = 0;  // rows per block; 0: sized per step from the rows in flight
    int64_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> pending;
    std::map<int64_t, Request> reqs;
    int64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> engines;
    std::atomic<int64_t> steps{0}, peak_active{0}, completed{0};
    std::atomic<int64_t> pool_peak{0};
    cudaMemPool_t pool = nullptr;

    void finish(Request &r, int status, const char *msg) {
        memset(&r.info, 0, sizeof r.info);
        r.info.status = status;
        r.info.alpha0 = __builtin_nan("");
        r.error = msg ? msg : "";
        r.started = r.finished = Clock::now();
        r.done = true;
    }

    void engine_loop();
};

// One engine: its stream, slots and the step pipeline.
void Server::engine_loop() {
    cudaSetDevice(device);
    // classic systems step on `st`, pipelined ones on `side` (forked after the
    // step's task list is copied, joined before its scalars are read back)
    cudaStream_t st = nullptr, side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) return;
    const int S = slots;
    const size_t cb = step_ctx_bytes();
    char *d_ctx = nullptr, *h_ctx = nullptr;
    SolverState *d_state = nullptr, *h_state = nullptr, *h_status = nullptr;
    DotScratch *d_scr = nullptr;
    StepTask *d_tasks[RING] = {}, *h_tasks[RING] = {};
    size_t cap_tasks[RING] = {};
    cudaEvent_t ev_step[RING] = {};
    bool ok = cudaMalloc(&d_ctx, S * cb) == cudaSuccess && cudaMalloc(&d_state, S * sizeof(SolverState)) == cudaSuccess &&
              cudaMalloc(&d_scr, S * sizeof(DotScratch)) == cudaSuccess &&
              cudaMemset(d_scr, 0, S * sizeof(DotScratch)) == cudaSuccess &&
              cudaMallocHost(&h_ctx, S * cb) == cudaSuccess &&
              cudaMallocHost(&h_state, S * sizeof(SolverState)) == cudaSuccess &&
              cudaMallocHost(&h_status, (size_t)RING * S * sizeof(SolverState)) == cudaSuccess;
    for (int k = 0; ok && k < RING; k++) ok = cudaEventCreateWithFlags(&ev_step[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) == cudaSuccess;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    ok = ok && cudaDeviceSynchronize() == cudaSuccess;

    struct Slot {
        int64_t ticket = -1;  // -1: free
        int variant = 0;
        int32_t maxit = 0, iters = 0;
        int64_t n = 0, bytes = 0;
        int64_t admit_step = -1, final_step = -1, last_step = -1;
        void *mem = nullptr;
    };
    std::vector<Slot> slot((size_t)S);
    int64_t step = 0, read_step = -1;  // steps enqueued; last step whose scalars were read
    int active = 0;
    std::vector<StepTask> tasks;
    std::vector<int> fresh;

    // rows per block of this step: the server's fixed size, or (0) one sized from
    // the rows in flight for about four waves of blocks (1024..65536 rows)
    int64_t rows = seg_rows > 0 ? seg_rows : 8192;
    auto add_tasks = [&](int s, std::vector<StepTask> &out) {
        const int64_t n = slot[(size_t)s].n;
        const int nblk = (int)((n + rows - 1) / rows);
        for (int b = 0; b < nblk; b++)
            out.push_back(StepTask{s, nblk, (int64_t)b * rows, std::min(n, (int64_t)(b + 1) * rows)});
    };
    auto fail_all = [&](const char *msg) {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &sl : slot)
            if (sl.ticket >= 0) {
                Request &r = reqs[sl.ticket];
                finish(r, RBS_ECUDA, msg);
                in_use -= sl.bytes;
                sl.ticket = -1;
            }
        cv_done.notify_all();
    };

    // read back the scalars of step j and retire what has stopped
    auto read = [&](int64_t j) {
        const SolverState *snap = h_status + (size_t)(j % RING) * S;
        for (int s = 0; s < S; s++) {
            Slot &sl = slot[(size_t)s];
            if (sl.ticket < 0 || sl.admit_step > j) continue;
            const SolverState &q = snap[s];
            const bool last = sl.final_step >= 0 && j >= sl.final_step;
            if (!q.done && !last) continue;
            rbs_info I;
            memset(&I, 0, sizeof I);
            I.iters = q.iter;
            I.status = q.status;
            I.converged = (q.status == RBS_OK && !(q.tau > q.tau_max)) ? 1 : 0;
            I.tau0 = q.tau0;
            I.tau_final = q.tau;
            I.rho0 = q.rho0;
            I.tau_max = q.tau_max;
            I.alpha0 = sl.variant == RBS_PIPELINED ? q.alpha0 : __builtin_nan("");
            I.mu0 = sl.variant == RBS_PIPELINED ? q.mu0 : 0.0;
            cudaFreeAsync(sl.mem, st);  // after every enqueued step that refers to it
            {
                std::lock_guard<std::mutex> lk(mu);
                Request &r = reqs[sl.ticket];
                r.info = I;
                if (q.status == RBS_EINVAL) r.error = "the system failed its CSR structure or diagonal check";
                r.finished = Clock::now();
                r.finish_step = j;
                r.done = true;
                in_use -= sl.bytes;
                completed++;
            }
            sl.ticket = -1;  // reusable once read_step >= last_step
            active--;
            cv_done.notify_all();
        }
        read_step = j;
    };

    while (ok) {
        // ---- admission: pending requests into free slots, within the budget
        fresh.clear();
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active == 0 && step - 1 == read_step)
                cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
            if (stopping && pending.empty() && active == 0 && step - 1 == read_step) break;
            int s = 0;
            while (!pending.empty()) {
                while (s < S && (slot[(size_t)s].ticket >= 0 || slot[(size_t)s].last_step > read_step)) s++;
                if (s >= S) break;
                Request &r = reqs[pending.front()];
                if (active + (int)fresh.size() > 0 && in_use + r.bytes > budget) break;
                pending.pop_front();
                in_use += r.bytes;
                r.started = Clock::now();
                r.admit_step = step;
                r.active_at_admit = active;
                Slot &sl = slot[(size_t)s];
                sl.ticket = r.ticket;
                sl.variant = r.sys.variant;
                sl.maxit = r.sys.maxit;
                sl.iters = 0;
                sl.n = r.sys.A.n;
                sl.bytes = r.bytes;
                sl.admit_step = step;
                sl.final_step = r.sys.maxit == 0 ? step : -1;
                sl.last_step = step;
                fresh.push_back(s);
                s++;
            }
        }
        for (int s : fresh) {
            Slot &sl = slot[(size_t)s];
            const rbs_system sys = [&] {
                std::lock_guard<std::mutex> lk(mu);
                return reqs[sl.ticket].sys;
            }();
            const int64_t stride = stride_of(sl.n);
            if (cudaMallocFromPoolAsync(&sl.mem, (size_t)stride * 8 * nvec_of(sl.variant), pool, st) != cudaSuccess) {
                ok = false;
                break;
            }
            double *v[16];
            for (int k = 0; k < nvec_of(sl.variant); k++) v[k] = (double *)sl.mem + (size_t)k * stride;
            SolverVecs V;
            memset(&V, 0, sizeof V);
            V.x = sys.x;
            V.r = v[0]; V.r0 = v[1]; V.ph = v[2]; V.s = v[3]; V.q = v[4]; V.qh = v[5]; V.y = v[6]; V.invd = v[7];
            if (sl.variant == RBS_CLASSIC) {
                V.p = v[8];
            } else {
                V.rh = v[8]; V.w = v[9]; V.wh = v[10]; V.t = v[11]; V.sh = v[12]; V.z = v[13]; V.zh = v[14]; V.v = v[15];
            }
            CSRArgs A{sys.A.n, sys.A.nnz, sys.A.rowptr, sys.A.col, sys.A.val};
            step_ctx_make(h_ctx + (size_t)s * cb, A, V, sys.b, sys.x0, sys.jacobi_diag, d_state + s, d_scr + s, nullptr);
            SolverState &h = h_state[s];
            memset(&h, 0, sizeof h);
            h.tol = sys.tol;
            h.maxit = sys.maxit;
            h.variant = sys.variant;
            // the pinned entries of slot s are rewritten only when s is reused, after
            // every step that read them has completed
            ok = ok && cudaMemcpyAsync(d_ctx + (size_t)s * cb, h_ctx + (size_t)s * cb, cb, cudaMemcpyHostToDevice, st) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(d_state + s, &h, sizeof h, cudaMemcpyHostToDevice, st) == cudaSuccess;
            active++;
        }
        if (!ok) break;
        if (active == 0) {  // nothing in flight: read back what is left, then wait
            if (step - 1 > read_step) {
                cudaEventSynchronize(ev_step[(step - 1) % RING]);
                for (int64_t j = read_step + 1; j < step; j++) read(j);
            }
            continue;
        }
        {
            int64_t pool_used = 0;
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &pool_used);
            if (pool_used > pool_peak.load()) pool_peak = pool_used;
        }
        // ---- this step's task lists: admissions, then one iteration of each variant
        if (seg_rows <= 0) {
            int64_t flight = 0;
            for (auto &sl : slot)
                if (sl.ticket >= 0) flight += sl.n;
            const int64_t waves = 4LL * sms * 3;
            rows = std::max<int64_t>(1024, std::min<int64_t>(65536, (flight + waves - 1) / waves));
            rows = (rows + 63) / 64 * 64;
        }
        tasks.clear();
        int off[3];  // admissions: classic tasks [off[0], off[1]), pipelined [off[1], off[2])
        for (int var = 0; var < 2; var++) {
            off[var] = (int)tasks.size();
            for (int s : fresh)
                if (slot[(size_t)s].variant == var) add_tasks(s, tasks);
        }
        off[2] = (int)tasks.size();
        int it_off[2], it_cnt[2];
        for (int var = 0; var < 2; var++) {
            it_off[var] = (int)tasks.size();
            for (int s = 0; s < S; s++) {
                Slot &sl = slot[(size_t)s];
                if (sl.ticket < 0 || sl.variant != var || sl.final_step >= 0) continue;
                add_tasks(s, tasks);
                sl.iters++;
                sl.last_step = step;
                if (sl.iters >= sl.maxit) sl.final_step = step;
            }
            it_cnt[var] = (int)tasks.size() - it_off[var];
        }
        if (active > peak_active.load()) peak_active = active;
        const int ring = (int)(step % RING);
        if (!tasks.empty()) {
            if (cap_tasks[ring] < tasks.size()) {
                cudaEventSynchronize(ev_step[ring]);
                if (h_tasks[ring]) cudaFreeHost(h_tasks[ring]);
                if (d_tasks[ring]) cudaFreeAsync(d_tasks[ring], st);
                size_t c = std::max<size_t>(tasks.size() * 2, 1024);
                ok = cudaMallocHost(&h_tasks[ring], c * sizeof(StepTask)) == cudaSuccess &&
                     cudaMallocAsync(&d_tasks[ring], c * sizeof(StepTask), st) == cudaSuccess;
                cap_tasks[ring] = ok ? c : 0;
                if (!ok) break;
            } else {
                cudaEventSynchronize(ev_step[ring]);  // the copy that last read this pinned buffer is done
            }
            memcpy(h_tasks[ring], tasks.data(), tasks.size() * sizeof(StepTask));
            ok = cudaMemcpyAsync(d_tasks[ring], h_tasks[ring], tasks.size() * sizeof(StepTask),
                                 cudaMemcpyHostToDevice, st) == cudaSuccess;
            const StepTask *T = d_tasks[ring];
            const bool pipe = off[2] > off[1] || it_cnt[1] > 0;
            if (pipe) {
                ok = ok && cudaEventRecord(ev_fork, st) == cudaSuccess &&
                     cudaStreamWaitEvent(side, ev_fork, 0) == cudaSuccess;
            }
            for (int var = 0; var < 2 && ok; var++) {
                cudaStream_t sv = var == RBS_CLASSIC ? st : side;
                if (off[var + 1] > off[var])
                    ok = step_admit(d_ctx, T + off[var], off[var + 1] - off[var], var, sv) == cudaSuccess;
                if (ok && it_cnt[var] > 0)
                    ok = step_iteration(d_ctx, T + it_off[var], it_cnt[var], var, sv) == cudaSuccess;
            }
            if (pipe) {
                ok = ok && cudaEventRecord(ev_join, side) == cudaSuccess &&
                     cudaStreamWaitEvent(st, ev_join, 0) == cudaSuccess;
            }
        }
        ok = ok && cudaMemcpyAsync(h_status + (size_t)ring * S, d_state, S * sizeof(SolverState),
                                   cudaMemcpyDeviceToHost, st) == cudaSuccess;
        ok = ok && cudaEventRecord(ev_step[ring], st) == cudaSuccess;
        if (!ok) break;
        step++;
        steps++;
        // ---- read back finished steps (at most DEPTH steps ahead of the reads)
        while (read_step < step - 1) {
            const int64_t j = read_step + 1;
            if (step - 1 - read_step > DEPTH) {
                if (cudaEventSynchronize(ev_step[j % RING]) != cudaSuccess) {
                    ok = false;
                    break;
                }
            } else if (cudaEventQuery(ev_step[j % RING]) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            read(j);
        }
    }
    if (!ok) fail_all("the serving engine met a CUDA error");
    cudaStreamSynchronize(side);
    cudaStreamSynchronize(st);
    for (auto &sl : slot)
        if (sl.mem && sl.ticket >= 0) cudaFreeAsync(sl.mem, st);
    for (int k = 0; k < RING; k++) {
        if (d_tasks[k]) cudaFreeAsync(d_tasks[k], st);
        if (h_tasks[k]) cudaFreeHost(h_tasks[k]);
        if (ev_step[k]) cudaEventDestroy(ev_step[k]);
    }
    cudaStreamSynchronize(st);
    cudaFree(d_ctx);
    cudaFree(d_state);
    cudaFree(d_scr);
    cudaFreeHost(h_ctx);
    cudaFreeHost(h_state);
    cudaFreeHost(h_status);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    cudaStreamSynchronize(side);
    cudaStreamDestroy(side);
    cudaStreamDestroy(st);
}

}  // namespace rbs

using namespace rbs;

extern "C" {

int rbs_server_create(int32_t engines, int32_t max_active, int64_t budget_bytes, int64_t rows_per_block,
                      rbs_server **out) {
    if (!out || engines < 1 || engines > 16 || max_active < 1 || max_active > 4096 || budget_bytes <= 0 ||
        rows_per_block < 0)
        return set_error(RBS_EINVAL, "rbs_server_create: bad argument");
    Server *s = new Server();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return set_error(RBS_ECUDA, "rbs_server_create: no current device");
    }
    s->slots = max_active;
    s->budget = budget_bytes;
    s->seg_rows = rows_per_block > 0 ? (rows_per_block + 63) / 64 * 64 : 0;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return set_error(RBS_ECUDA, "rbs_server_create: cudaMemPoolCreate failed");
    }
    // keep up to the budget reserved between steps; above it, memory goes back
    uint64_t keep = (uint64_t)budget_bytes;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int i = 0; i < engines; i++) s->engines.emplace_back([s] { s->engine_loop(); });
    *out = reinterpret_cast<rbs_server *>(s);
    return RBS_OK;
}

int rbs_server_submit(rbs_server *srv, const rbs_system *system, int64_t *ticket) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s || !system || !ticket) return set_error(RBS_EINVAL, "rbs_server_submit: bad argument");
    const char *why = bad_system(*system);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return set_error(RBS_EINVAL, "rbs_server_submit: server is stopping");
        Request r;
        memset(&r.info, 0, sizeof r.info);
        r.ticket = s->next_ticket++;
        r.sys = *system;
        r.bytes = state_bytes(*system);
        r.submitted = Clock::now();
        r.done = false;
        r.admit_step = r.finish_step = -1;
        r.active_at_admit = 0;
        s->reqs[r.ticket] = r;
        *ticket = r.ticket;
        if (why) {
            s->finish(s->reqs[r.ticket], RBS_EINVAL, why);
        } else {
            s->pending.push_back(r.ticket);
        }
    }
    if (why) s->cv_done.notify_all();
    else s->cv_work.notify_all();
    return RBS_OK;
}

static void fill_result(const Request &r, rbs_info *info, double *latency_s, double *queue_s) {
    if (!r.error.empty()) set_error(r.info.status, r.error.c_str());
    if (info) *info = r.info;
    if (latency_s) *latency_s = std::chrono::duration<double>(r.finished - r.submitted).count();
    if (queue_s) *queue_s = std::chrono::duration<double>(r.started - r.submitted).count();
}

int rbs_server_poll(rbs_server *srv, int64_t ticket, int32_t *done, rbs_info *info, double *latency_s,
                    double *queue_s) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s || !done) return set_error(RBS_EINVAL, "rbs_server_poll: bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(RBS_EINVAL, "rbs_server_poll: unknown ticket");
    *done = it->second.done ? 1 : 0;
    if (it->second.done) fill_result(it->second, info, latency_s, queue_s);
    return RBS_OK;
}

int rbs_server_wait(rbs_server *srv, int64_t ticket, rbs_info *info, double *latency_s, double *queue_s) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s) return set_error(RBS_EINVAL, "rbs_server_wait: bad argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(RBS_EINVAL, "rbs_server_wait: unknown ticket");
    s->cv_done.wait(lk, [&] { return s->reqs[ticket].done; });
    fill_result(s->reqs[ticket], info, latency_s, queue_s);
    return RBS_OK;
}

int rbs_server_request_stats(rbs_server *srv, int64_t ticket, rbs_request_stats *out) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s || !out) return set_error(RBS_EINVAL, "rbs_server_request_stats: bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(RBS_EINVAL, "rbs_server_request_stats: unknown ticket");
    const Request &r = it->second;
    out->admit_step = r.admit_step;
    out->finish_step = r.finish_step;
    out->active_at_admit = r.active_at_admit;
    out->done = r.done ? 1 : 0;
    return RBS_OK;
}

int rbs_server_stats(rbs_server *srv, rbs_server_counters *out) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s || !out) return set_error(RBS_EINVAL, "rbs_server_stats: bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->steps = s->steps.load();
    out->completed = s->completed.load();
    out->peak_active = s->peak_active.load();
    out->pending = (int64_t)s->pending.size();
    out->budget_in_use = s->in_use;
    out->pool_reserved_peak = s->pool_peak.load();
    int64_t cur = 0;
    cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemCurrent, &cur);
    out->pool_reserved = cur;
    return RBS_OK;
}

int rbs_server_destroy(rbs_server *srv) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s) return RBS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->engines) t.join();
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return RBS_OK;
}

}  // extern "C"
