// Serving loop (the SCBA-style request stream): requests from independent SCBA iterations
// (Section 2 iterates GF -> SSE until convergence) arrive at any time; each names a plan and
// device buffers that the caller keeps resident between iterations.  A server thread
// admits pending requests in arrival order while the admitted working sets fit the memory
// budget and the in-flight cap, and launches every admitted-but-not-started request as one
// persistent batched round.  The server owns kSlots streams, each with its own device
// status word and work counter; a round is launched on a stream that no running round
// uses, so a round formed from new arrivals starts while older rounds drain: continuous
// batching rather than one queue drained at a time.  Each round copies its status word to
// pinned host memory behind its kernels and records an event; the server thread polls the
// events and never synchronises a stream.  sse_poll reports status and timestamps.
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

constexpr int kSlots = 2;  // streams, and so rounds in flight at once

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kPending = 0, kAdmitted = 1, kRunning = 2, kDone = 3 };

struct Request {
    sse_plan_t *plan = nullptr;
    sse_io io{};
    uint64_t bytes = 0;  // G, Dt and Sigma of the requested signs (the plan's workspace is counted per plan)
    double t_submit = 0, t_start = 0, t_end = 0;
    sse_status status = SSE_NOT_READY;
    ReqState state = kPending;
    int round_size = 0;
};

// One stream with what a round on it needs: the device status word and work counter
// (d_words[0], d_words[1]), the pinned host copy of the status word, the completion event.
struct Slot {
    cudaStream_t stream = nullptr;
    int32_t *d_words = nullptr;
    volatile int32_t *h_status = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
};

struct Round {
    int slot = 0;
    std::vector<uint64_t> tickets;
};

}  // namespace

struct sse_server_s {
    std::mutex mu;
    std::condition_variable cv;
    std::thread thread;
    bool stop = false;        // shutdown requested: admit nothing more
    bool thread_done = false;  // the server thread has left its loop
    int device = 0;
    uint64_t budget = 0, inflight_bytes = 0;
    int max_inflight = 1, inflight = 0;
    uint32_t wait_limit_ms = 1000;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::unordered_map<const sse_plan_t *, int> plan_refs;  // admitted requests per plan
    std::vector<Round> running;
    Slot slots[kSlots];
    int32_t *d_words = nullptr;
    int32_t *h_words = nullptr;
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

// Device bytes the library holds for a plan (status word and tensor-core workspace).
uint64_t plan_bytes(const Plan &p) { return (uint64_t)p.workspace_bytes; }

// Bytes admitting request q adds to the working set: its buffers, plus its plan's
// workspace when no admitted request holds that plan yet.
uint64_t admit_bytes(const sse_server_s *s, const Request &q) {
    auto it = s->plan_refs.find(q.plan);
    const bool held = it != s->plan_refs.end() && it->second > 0;
    return q.bytes + (held ? 0 : plan_bytes(*plan_core(q.plan)));
}

void admit(sse_server_s *s, Request &q) {
    s->inflight_bytes += admit_bytes(s, q);
    s->plan_refs[q.plan] += 1;
    s->inflight += 1;
    q.state = kAdmitted;
}

// Undo admit() once the request is final.
void release(sse_server_s *s, Request &q) {
    s->inflight_bytes -= q.bytes;
    auto it = s->plan_refs.find(q.plan);
    if (it != s->plan_refs.end() && --it->second == 0) {
        s->inflight_bytes -= plan_bytes(*plan_core(q.plan));
        s->plan_refs.erase(it);
    }
    s->inflight -= 1;
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
        release(s, q);
    }
    s->slots[r.slot].busy = false;
}

// Launch the admitted requests in `group` as one round on a free slot.  Called with the
// lock held; releases it around the CUDA calls (only this thread launches rounds, and
// running requests are touched by nobody else).
void launch_round(sse_server_s *s, std::unique_lock<std::mutex> &lock, std::vector<uint64_t> &group) {
    int si = 0;
    while (si < kSlots && s->slots[si].busy) ++si;
    if (si == kSlots) return;  // the caller keeps at most kSlots rounds running
    Slot &slot = s->slots[si];
    slot.busy = true;
    Round r;
    r.slot = si;
    r.tickets = group;
    std::vector<Plan *> plans;
    std::vector<double> slots_per_atom;
    std::vector<sse_io> ios;
    for (uint64_t tk : group) {
        Request &q = s->reqs[tk];
        q.state = kRunning;
        q.round_size = (int)group.size();
        plans.push_back(plan_core(q.plan));
        slots_per_atom.push_back(plan_slots_per_atom(q.plan));
        ios.push_back(q.io);
    }
    s->rounds_launched += 1;
    lock.unlock();
    cudaStream_t st = slot.stream;
    sse_status rs = SSE_OK;
    cudaError_t e = cudaMemsetAsync(slot.d_words, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) rs = cuda_fail(e, "clear the round's status word");
    if (rs == SSE_OK)
        rs = run_batch(plans.data(), slots_per_atom.data(), ios.data(), (int)plans.size(), st, slot.d_words, nullptr,
                       nullptr, /*allow_tune=*/false, slot.d_words + 1);
    if (rs == SSE_OK) {
        e = cudaMemcpyAsync((void *)slot.h_status, slot.d_words, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(slot.done, st);
        if (e != cudaSuccess) rs = cuda_fail(e, "record the round's completion");
    }
    lock.lock();
    // t_start: the round's kernels are enqueued (set only now, so a caller that sees it knows
    // the launch has been issued)
    const double t_launched = now_ms();
    for (uint64_t tk : group) s->reqs[tk].t_start = t_launched;
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
        // completions: a round is done when its event has fired; its status word (copied to
        // pinned host memory behind the kernels) then holds every expired device wait
        for (size_t i = 0; i < s->running.size();) {
            Slot &slot = s->slots[s->running[i].slot];
            cudaError_t e = cudaEventQuery(slot.done);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            sse_status st = SSE_OK;
            if (e != cudaSuccess) st = cuda_fail(e, "round");
            else if (*slot.h_status & kStatusBounds) st = SSE_E_BOUNDS;
            else if (*slot.h_status != 0) st = SSE_E_TIMEOUT;
            finish_round(s, s->running[i], st);
            s->running.erase(s->running.begin() + (long)i);
        }
        if (s->stop && s->running.empty()) break;
        if (!s->stop) {
            // admission in arrival order while the working sets fit
            while (!s->pending.empty()) {
                Request &q = s->reqs[s->pending.front()];
                if (s->inflight >= s->max_inflight || s->inflight_bytes + admit_bytes(s, q) > s->budget) break;
                admit(s, q);
                s->pending.pop_front();
            }
            // one round per compatible group of admitted requests while a stream is free; a
            // plan runs in one round at a time and once per round (its workspace is its own)
            while ((int)s->running.size() < kSlots && !s->stop) {
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
                launch_round(s, lock, group);
            }
        }
        s->cv.wait_for(lock, std::chrono::microseconds(s->running.empty() ? 2000 : 50));
    }
    s->thread_done = true;
}

// Cancel what has not started and stop admitting; requests that never ran end with
// SSE_E_CANCELLED and stay pollable.  Called with the lock held.
void cancel_unstarted(sse_server_s *s) {
    s->stop = true;
    const double t = now_ms();
    for (uint64_t tk : s->pending) {
        Request &q = s->reqs[tk];
        q.state = kDone;
        q.status = SSE_E_CANCELLED;
        q.t_end = t;
    }
    s->pending.clear();
    for (auto &kv : s->reqs)
        if (kv.second.state == kAdmitted) {
            kv.second.state = kDone;
            kv.second.status = SSE_E_CANCELLED;
            kv.second.t_end = t;
            release(s, kv.second);
        }
}

void free_server(sse_server_s *s) {
    for (Slot &sl : s->slots) {
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->d_words) cudaFree(s->d_words);
    if (s->h_words) cudaFreeHost(s->h_words);
    delete s;
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
    cudaError_t e = cudaMalloc(&s->d_words, 2 * kSlots * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_words, kSlots * sizeof(int32_t), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMemset(s->d_words, 0, 2 * kSlots * sizeof(int32_t));
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        Slot &sl = s->slots[i];
        sl.d_words = s->d_words + 2 * i;
        sl.h_status = s->h_words + i;
        *sl.h_status = 0;
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        sse_status rs = cuda_fail(e, "create the server's streams and status words");
        cudaGetLastError();
        free_server(s);
        return rs;
    }
    try {
        s->thread = std::thread(server_loop, s);
    } catch (...) {
        free_server(s);
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
    if (bytes + plan_bytes(*p) > s->budget)
        return set_error("request needs %llu bytes (buffers and plan workspace), budget is %llu",
                         (unsigned long long)(bytes + plan_bytes(*p)), (unsigned long long)s->budget),
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

SSE_API sse_status sse_server_shutdown(sse_server_t *s) {
    if (!s) return set_error("server is NULL"), SSE_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        cancel_unstarted(s);
    }
    s->cv.notify_one();
    // running rounds drain; give them the configured bound, then stop waiting
    const double t0 = now_ms();
    while (true) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->thread_done) return SSE_OK;
        }
        if (now_ms() - t0 > s->wait_limit_ms) {
            set_error("rounds still running after %u ms at shutdown", s->wait_limit_ms);
            return SSE_E_TIMEOUT;
        }
        s->cv.notify_one();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

SSE_API sse_status sse_server_destroy(sse_server_t *s) {
    if (!s) return SSE_OK;
    const sse_status rs = sse_server_shutdown(s);
    if (rs == SSE_OK) {
        s->thread.join();
        free_server(s);
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
