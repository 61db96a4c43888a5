// Serving runtime: a request loop with continuous batching.
//
// Clients submit solves (rbs_system, device data) at any time. Worker threads,
// each owning its own CUDA stream and so its own library workspace, take the
// pending requests that fit the memory budget (Krylov state of in-flight
// requests). A large system (n >= solo_n) runs alone with the whole-GPU
// per-step solver; consecutive small ones run together as one batched cluster
// launch. Requests that arrive while others run are admitted as soon as a
// worker and budget free up, and work on different streams overlaps on the
// device. Each answer is bitwise the one a solve of that system alone gives
// (both paths guarantee it). Latency is measured from submission to completion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "launch.h"
#include "rbs.h"

namespace rbs {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    rbs_system sys;
    int64_t bytes;  // device memory the solve keeps while in flight
    Clock::time_point submitted, started, finished;
    rbs_info info;
    bool done;
    int batch_size;
    std::string error;  // message of a call that failed as a whole
};

int64_t state_bytes(const rbs_system &s) {
    const int64_t stride = (s.A.n + 31) / 32 * 32;
    return stride * 8 * (s.variant == RBS_PIPELINED ? 17 : 9);
}

}  // namespace

struct Server {
    int device = 0;
    int max_batch = 8;
    int64_t solo_n = 100000;
    int64_t budget = 0, in_flight = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> pending;
    std::map<int64_t, Request> reqs;
    int64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
    std::atomic<int64_t> completed{0};

    void worker_loop() {
        cudaSetDevice(device);
        cudaStream_t stream = nullptr;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return;
        std::vector<int64_t> mine;
        std::vector<rbs_system> sys;
        std::vector<rbs_info> infos;
        for (;;) {
            mine.clear();
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    if (stopping) return true;
                    if (pending.empty()) return false;
                    const Request &r = reqs[pending.front()];
                    return in_flight == 0 || in_flight + r.bytes <= budget;
                });
                if (stopping && pending.empty()) break;
                // admit in arrival order while the budget allows (always at least one
                // request when nothing is in flight, so an oversized one still runs);
                // a large system goes alone, small ones are batched together
                while (!pending.empty() && (int)mine.size() < max_batch) {
                    Request &r = reqs[pending.front()];
                    if (in_flight > 0 && in_flight + r.bytes > budget) break;
                    const bool large = r.sys.A.n >= solo_n;
                    if (large && !mine.empty()) break;
                    in_flight += r.bytes;
                    r.started = Clock::now();
                    mine.push_back(r.ticket);
                    pending.pop_front();
                    if (large) break;
                }
                sys.clear();
                for (int64_t t : mine) sys.push_back(reqs[t].sys);
            }
            if (mine.empty()) continue;
            infos.assign(mine.size(), rbs_info{});
            int rc;
            if (mine.size() == 1 && sys[0].A.n >= solo_n) {
                const rbs_system &q = sys[0];
                rbs_opts o{};
                rc = rbs_solve_ex(&q.A, q.b, q.x0, q.jacobi_diag, q.tol, q.maxit, q.variant, &o, q.x, &infos[0],
                                  nullptr, nullptr, stream);
            } else {
                rc = rbs_solve_batched((int32_t)mine.size(), sys.data(), infos.data(), nullptr, stream);
            }
            // a call that failed as a whole leaves its requests unsolved: they
            // report its status (per-system statuses are already in infos)
            const char *msg = rc ? rbs_last_error() : "";
            {
                std::lock_guard<std::mutex> lk(mu);
                const auto now = Clock::now();
                for (size_t i = 0; i < mine.size(); i++) {
                    Request &r = reqs[mine[i]];
                    r.info = infos[i];
                    if (rc && r.info.status == RBS_OK && r.info.iters == 0) {
                        r.info.status = rc;
                        r.error = msg;
                    }
                    r.finished = now;
                    r.done = true;
                    r.batch_size = (int)mine.size();
                    in_flight -= r.bytes;
                }
                completed += (int64_t)mine.size();
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        release_stream_workspace(stream);
        cudaStreamDestroy(stream);
    }
};

}  // namespace rbs

using namespace rbs;

extern "C" {

int rbs_server_create(int32_t workers, int32_t max_batch, int64_t budget_bytes, int64_t solo_n,
                      rbs_server **out) {
    if (!out || workers < 1 || workers > 64 || max_batch < 1 || budget_bytes <= 0 || solo_n < 0)
        return set_error(RBS_EINVAL, "rbs_server_create: bad argument");
    Server *s = new Server();
    s->solo_n = solo_n;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return set_error(RBS_ECUDA, "rbs_server_create: no current device");
    }
    s->max_batch = max_batch;
    s->budget = budget_bytes;
    for (int i = 0; i < workers; i++) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = reinterpret_cast<rbs_server *>(s);
    return RBS_OK;
}

int rbs_server_submit(rbs_server *srv, const rbs_system *system, int64_t *ticket) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s || !system || !ticket) return set_error(RBS_EINVAL, "rbs_server_submit: bad argument");
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
        r.batch_size = 0;
        s->reqs[r.ticket] = r;
        s->pending.push_back(r.ticket);
        *ticket = r.ticket;
    }
    s->cv_work.notify_one();
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

int rbs_server_destroy(rbs_server *srv) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s) return RBS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
    return RBS_OK;
}

}  // extern "C"
