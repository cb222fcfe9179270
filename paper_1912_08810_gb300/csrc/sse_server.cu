// Serving loop (the SCBA-style request stream): requests from independent SCBA iterations
// (Section 2 iterates GF -> SSE until convergence) arrive at any time; each names a plan and
// device buffers that the caller keeps resident between iterations.  A server thread
// admits pending requests in arrival order while the admitted working sets fit the memory
// budget and the in-flight cap, and launches every admitted-but-not-started request as one
// persistent batched round on one of two streams.  Rounds alternate streams, so a round
// formed from new arrivals starts while the previous one is still draining: continuous
// batching rather than one queue drained at a time.  Completion is detected with events;
// sse_poll reports status and timestamps.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sse_internal.h"

using namespace sse;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kPending = 0, kAdmitted = 1, kRunning = 2, kDone = 3 };

struct Request {
    sse_plan_t *plan = nullptr;
    sse_io io{};
    uint64_t bytes = 0;
    double t_submit = 0, t_start = 0, t_end = 0;
    sse_status status = SSE_NOT_READY;
    ReqState state = kPending;
    int round_size = 0;
};

struct Round {
    cudaEvent_t done = nullptr;
    int stream = 0;
    std::vector<uint64_t> tickets;
    double t_launch = 0;
};

}  // namespace

struct sse_server_s {
    std::mutex mu;
    std::condition_variable cv;
    std::thread thread;
    bool stop = false;
    int device = 0;
    uint64_t budget = 0, inflight_bytes = 0;
    int max_inflight = 1, inflight = 0;
    uint32_t wait_limit_ms = 1000;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Round> running;
    cudaStream_t streams[2] = {nullptr, nullptr};
    int next_stream = 0;
    uint64_t rounds_launched = 0;
};

namespace sse {
// Plan internals needed here (defined in sse_abi.cu).
Plan *plan_core(sse_plan_t *p);
double plan_slots_per_atom(const sse_plan_t *p);
sse_status plan_check_io(sse_plan_t *p, const sse_io *io);
}  // namespace sse

namespace {

// Device bytes a request keeps resident: G, Dt and Sigma of each requested sign.
uint64_t request_bytes(const Plan &p, const sse_io &io) {
    const size_t eb = elem_bytes(p.geo.dtype);
    const uint64_t per_sign = (uint64_t)(2 * g_elems(p.d) + d_elems(p.d)) * eb;
    return per_sign * ((io.S_gt != nullptr) + (io.S_lt != nullptr));
}

// Two plans can share a persistent launch when the compile-time shape and the shared
// launch parameters agree.
bool compatible(const Plan &a, const Plan &b) {
    return a.d.nkz == b.d.nkz && a.d.nw == b.d.nw && a.d.omega_first == b.d.omega_first &&
           a.geo.dtype == b.geo.dtype;
}

void finish_round(sse_server_s *s, Round &r, sse_status st) {
    const double t = now_ms();
    for (uint64_t tk : r.tickets) {
        auto it = s->reqs.find(tk);
        if (it == s->reqs.end()) continue;
        Request &q = it->second;
        q.state = kDone;
        q.t_end = t;
        if (q.status == SSE_NOT_READY) q.status = st;
        s->inflight_bytes -= q.bytes;
        s->inflight -= 1;
    }
    if (r.done) cudaEventDestroy(r.done);
    r.done = nullptr;
}

// Launch every admitted request of one compatible group as a round.  Called with the lock.
void launch_round(sse_server_s *s, std::vector<uint64_t> &group) {
    Round r;
    r.stream = s->next_stream;
    s->next_stream ^= 1;
    r.tickets = group;
    r.t_launch = now_ms();
    std::vector<Plan *> plans;
    std::vector<double> slots;
    std::vector<sse_io> ios;
    for (uint64_t tk : group) {
        Request &q = s->reqs[tk];
        q.state = kRunning;
        q.t_start = r.t_launch;
        q.round_size = (int)group.size();
        plans.push_back(plan_core(q.plan));
        slots.push_back(plan_slots_per_atom(q.plan));
        ios.push_back(q.io);
    }
    cudaStream_t st = s->streams[r.stream];
    sse_status rs = run_batch(plans.data(), slots.data(), ios.data(), (int)plans.size(), st, nullptr, nullptr,
                              /*allow_tune=*/false);
    if (rs == SSE_OK) {
        cudaError_t e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r.done, st);
        if (e != cudaSuccess) rs = cuda_fail(e, "record round event");
    }
    s->rounds_launched += 1;
    if (rs != SSE_OK) {
        finish_round(s, r, rs);
        return;
    }
    s->running.push_back(r);
}

void server_loop(sse_server_s *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        // completions
        for (size_t i = 0; i < s->running.size();) {
            cudaError_t e = cudaEventQuery(s->running[i].done);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            sse_status st = SSE_OK;
            if (e != cudaSuccess) st = cuda_fail(e, "round");
            // a device wait that expired is recorded in the first plan's status word
            if (st == SSE_OK) {
                Request &q0 = s->reqs[s->running[i].tickets[0]];
                cudaStream_t rst = s->streams[s->running[i].stream];
                int32_t v = 0;
                if (cudaMemcpyAsync(&v, plan_core(q0.plan)->d_status, sizeof v, cudaMemcpyDeviceToHost, rst) ==
                        cudaSuccess &&
                    cudaStreamSynchronize(rst) == cudaSuccess && v != 0) {
                    cudaMemsetAsync(plan_core(q0.plan)->d_status, 0, sizeof v, rst);
                    st = SSE_E_TIMEOUT;
                }
            }
            finish_round(s, s->running[i], st);
            s->running.erase(s->running.begin() + (long)i);
        }
        if (s->stop && s->running.empty()) break;
        // admission in arrival order while the working sets fit
        if (!s->stop) {
            while (!s->pending.empty()) {
                Request &q = s->reqs[s->pending.front()];
                if (s->inflight >= s->max_inflight || s->inflight_bytes + q.bytes > s->budget) break;
                q.state = kAdmitted;
                s->inflight += 1;
                s->inflight_bytes += q.bytes;
                s->pending.pop_front();
            }
            // one round per compatible group of admitted requests, at most two rounds queued;
            // a plan runs in one round at a time and once per round (its workspace is its own)
            while (s->running.size() < 2) {
                std::vector<uint64_t> group;
                std::vector<const sse_plan_t *> busy;
                for (const Round &r : s->running)
                    for (uint64_t tk : r.tickets) busy.push_back(s->reqs[tk].plan);
                const Plan *ref = nullptr;
                for (auto &kv : s->reqs) {
                    Request &q = kv.second;
                    if (q.state != kAdmitted) continue;
                    if (std::find(busy.begin(), busy.end(), q.plan) != busy.end()) continue;
                    const Plan *p = plan_core(q.plan);
                    if (!ref) ref = p;
                    if (compatible(*ref, *p)) {
                        group.push_back(kv.first);
                        busy.push_back(q.plan);
                    }
                }
                if (group.empty()) break;
                std::sort(group.begin(), group.end());  // arrival order
                launch_round(s, group);
            }
        }
        s->cv.wait_for(lock, std::chrono::microseconds(s->running.empty() ? 2000 : 50));
    }
}

}  // namespace

extern "C" {

SSE_API sse_status sse_server_create(uint64_t mem_budget_bytes, int32_t max_inflight, uint32_t wait_limit_ms,
                                     sse_server_t **out) {
    if (!out || mem_budget_bytes == 0 || max_inflight <= 0)
        return set_error("bad server arguments"), SSE_E_INVALID_ARG;
    *out = nullptr;
    sse_server_s *s = new (std::nothrow) sse_server_s();
    if (!s) return set_error("host allocation failed"), SSE_E_OUT_OF_MEMORY;
    s->budget = mem_budget_bytes;
    s->max_inflight = max_inflight;
    s->wait_limit_ms = wait_limit_ms ? wait_limit_ms : 1000;
    cudaGetDevice(&s->device);
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (i == 1) cudaStreamDestroy(s->streams[0]);
            delete s;
            return cuda_fail(e, "create server stream");
        }
    }
    try {
        s->thread = std::thread(server_loop, s);
    } catch (...) {
        cudaStreamDestroy(s->streams[0]);
        cudaStreamDestroy(s->streams[1]);
        delete s;
        return set_error("could not start the server thread"), SSE_E_OUT_OF_MEMORY;
    }
    *out = s;
    return SSE_OK;
}

SSE_API sse_status sse_submit(sse_server_t *s, sse_plan_t *plan, const sse_io *io, uint64_t *ticket) {
    if (!s || !plan || !io || !ticket) return set_error("NULL argument"), SSE_E_INVALID_ARG;
    const Plan *p = plan_core(plan);
    if (p->kernel_id != 1) return set_error("the server runs mixed-mode plans"), SSE_E_INVALID_ARG;
    sse_status st = plan_check_io(plan, io);
    if (st != SSE_OK) return st;
    if (!io->S_gt && !io->S_lt) return set_error("request computes no sign"), SSE_E_INVALID_ARG;
    const uint64_t bytes = request_bytes(*p, *io);
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return set_error("server is shutting down"), SSE_E_SHUTDOWN;
    if (bytes > s->budget)
        return set_error("request needs %llu bytes, budget is %llu", (unsigned long long)bytes,
                         (unsigned long long)s->budget),
               SSE_E_OVER_BUDGET;
    const uint64_t tk = s->next_ticket++;
    Request q;
    q.plan = plan;
    q.io = *io;
    q.bytes = bytes;
    q.t_submit = now_ms();
    s->reqs.emplace(tk, q);
    s->pending.push_back(tk);
    *ticket = tk;
    s->cv.notify_one();
    return SSE_OK;
}

SSE_API sse_status sse_poll(sse_server_t *s, uint64_t ticket, sse_result *out) {
    if (!s) return set_error("server is NULL"), SSE_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error("unknown ticket %llu", (unsigned long long)ticket), SSE_E_UNKNOWN_TICKET;
    Request &q = it->second;
    if (out) {
        out->status = q.status;
        out->t_submit_ms = q.t_submit;
        out->t_start_ms = q.t_start;
        out->t_end_ms = q.t_end;
        out->round_size = q.round_size;
    }
    if (q.state != kDone) return SSE_NOT_READY;
    const sse_status st = q.status;
    s->reqs.erase(it);
    return st;
}

SSE_API sse_status sse_server_destroy(sse_server_t *s) {
    if (!s) return SSE_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        // requests that never started are cancelled
        for (uint64_t tk : s->pending) {
            Request &q = s->reqs[tk];
            q.state = kDone;
            q.status = SSE_E_CANCELLED;
        }
        s->pending.clear();
        for (auto &kv : s->reqs)
            if (kv.second.state == kAdmitted) {
                kv.second.state = kDone;
                kv.second.status = SSE_E_CANCELLED;
                s->inflight -= 1;
                s->inflight_bytes -= kv.second.bytes;
            }
    }
    s->cv.notify_one();
    // running rounds drain; give them the configured bound, then stop waiting
    const double t0 = now_ms();
    sse_status rs = SSE_OK;
    while (true) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->running.empty()) break;
        }
        if (now_ms() - t0 > s->wait_limit_ms) {
            rs = SSE_E_TIMEOUT;
            set_error("rounds still running after %u ms at shutdown", s->wait_limit_ms);
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    if (rs == SSE_OK) {
        s->thread.join();
        cudaStreamDestroy(s->streams[0]);
        cudaStreamDestroy(s->streams[1]);
        delete s;
    } else {
        // the GPU still holds this server's work: keep the object alive (leaked) rather than
        // free streams and buffers under running kernels
        s->thread.detach();
    }
    return rs;
}

SSE_API sse_status sse_server_stats(sse_server_t *s, uint64_t *rounds, uint64_t *inflight_bytes, int32_t *inflight) {
    if (!s) return set_error("server is NULL"), SSE_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (rounds) *rounds = s->rounds_launched;
    if (inflight_bytes) *inflight_bytes = s->inflight_bytes;
    if (inflight) *inflight = s->inflight;
    return SSE_OK;
}

}  // extern "C"
