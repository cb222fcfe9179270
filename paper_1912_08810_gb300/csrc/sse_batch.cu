// Batched execution: many independent instances (uneven Na, NE, per-atom neighbour counts)
// in one persistent launch of the mixed kernel, with the work split chosen by a small
// exhaustive autotuner (in the spirit of the tile-size search of Section 3,
// "Communication Avoidance", which enumerates all feasible tilings).
//
// Tuned knobs: tiles per work unit (1 .. 16) and the order in which instances enter the
// work queue (as given, or longest unit first).  The first call for a batch shape times
// every candidate once on the caller's stream, on a sample of up to 8 instances spread over
// the size range, and keeps the fastest for the whole batch; the choice is cached
// in memory and, when SSE_AUTOTUNE_CACHE names a file, appended to that file and read back
// by later processes.  SSE_AUTOTUNE=0 skips tuning (tiles per unit 2, longest first).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "sse_internal.h"

struct sse_plan_s;  // defined in sse_abi.cu; plans are handled here through sse::Plan

namespace sse {
namespace {

struct Choice {
    int tpc;
    int lpt;
};

std::mutex g_mu;
std::unordered_map<unsigned long long, Choice> g_cache;
bool g_loaded = false;

unsigned long long fnv(unsigned long long h, long long v) {
    for (int i = 0; i < 8; ++i) {
        h ^= (unsigned long long)((v >> (8 * i)) & 0xff);
        h *= 1099511628211ull;
    }
    return h;
}

// Order-independent signature of a batch shape.
unsigned long long signature(Plan *const *plans, const sse_io *ios, int n) {
    std::vector<std::vector<long long>> rows;
    rows.reserve(n);
    for (int i = 0; i < n; ++i) {
        const Dims &d = plans[i]->d;
        rows.push_back({d.na, d.ne, d.nb, d.nqz, (long long)(ios[i].S_gt != nullptr) + (ios[i].S_lt != nullptr)});
    }
    std::sort(rows.begin(), rows.end());
    unsigned long long h = 1469598103934665603ull;
    const Dims &d0 = plans[0]->d;
    h = fnv(h, d0.nkz);
    h = fnv(h, d0.nw);
    h = fnv(h, d0.omega_first);
    h = fnv(h, plans[0]->geo.dtype);
    for (auto &r : rows)
        for (long long v : r) h = fnv(h, v);
    return h;
}

void load_cache_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("SSE_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    unsigned long long sig;
    int tpc, lpt;
    while (fscanf(f, "%llx %d %d", &sig, &tpc, &lpt) == 3)
        if (tpc >= 1 && tpc <= 1024) g_cache[sig] = Choice{tpc, lpt ? 1 : 0};
    fclose(f);
}

void save_choice(unsigned long long sig, Choice c) {
    const char *path = getenv("SSE_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%016llx %d %d\n", sig, c.tpc, c.lpt);
    fclose(f);
}

// Instance order: as given, or by decreasing work per unit (tiles per unit x valid slots
// per atom), so the longest units start first and the tail stays short.
std::vector<int> make_order(Plan *const *plans, const double *slots_per_atom, int n, int tpc, bool lpt) {
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if (lpt) {
        std::vector<double> cost(n);
        for (int i = 0; i < n; ++i) {
            const int te = plans[i]->tile_e > 0 ? plans[i]->tile_e : 1;
            const int ntiles = (plans[i]->d.ne + te - 1) / te;
            cost[i] = (double)std::min(tpc, ntiles) * slots_per_atom[i];
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    }
    return order;
}

}  // namespace

sse_status run_batch(Plan *const *plans, const double *slots_per_atom, const sse_io *ios, int n, cudaStream_t st,
                     int32_t *status, int *tpc_out, int *lpt_out, bool allow_tune, int32_t *queue_in) {
    if (n == 0) return SSE_OK;
    const unsigned long long sig = signature(plans, ios, n);
    Choice ch{2, 1};
    bool have = false;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        load_cache_locked();
        auto it = g_cache.find(sig);
        if (it != g_cache.end()) {
            ch = it->second;
            have = true;
        }
    }
    int32_t *queue = queue_in;
    cudaError_t e = cudaSuccess;
    if (!queue) {
        if (take_inject(SSE_INJECT_ALLOC_FAIL)) return set_error("injected allocation failure (work counter)"), SSE_E_OUT_OF_MEMORY;
        e = cudaMallocAsync((void **)&queue, sizeof(int32_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(work counter)");
    }
    sse_status rs = SSE_OK;
    const char *tune_env = getenv("SSE_AUTOTUNE");
    if (!have && allow_tune && !(tune_env && tune_env[0] == '0')) {
        // Exhaustive search over (tiles per unit, order), each candidate timed once on a
        // sample of at most kSample instances spread evenly over the batch sorted by size
        // (the whole batch when it is that small); one untimed warm run first.
        constexpr int kSample = 8;
        std::vector<int> idx(n);
        for (int i = 0; i < n; ++i) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](int x, int y) {
            return (long long)plans[x]->d.na * plans[x]->d.ne > (long long)plans[y]->d.na * plans[y]->d.ne;
        });
        std::vector<Plan *> sp;
        std::vector<double> ss;
        std::vector<sse_io> sio;
        const int m = n < kSample ? n : kSample;
        for (int x = 0; x < m; ++x) {
            const int i = idx[(long long)x * n / m];
            sp.push_back(plans[i]);
            ss.push_back(slots_per_atom[i]);
            sio.push_back(ios[i]);
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        const int tpcs[] = {1, 2, 4, 8, 16};
        {
            std::vector<int> order = make_order(sp.data(), ss.data(), m, 2, true);
            rs = launch_mixed_batch(sp.data(), sio.data(), order.data(), m, 2, queue, status, st);
        }
        for (int lpt = 0; lpt < 2 && rs == SSE_OK; ++lpt)
            for (int tpc : tpcs) {
                std::vector<int> order = make_order(sp.data(), ss.data(), m, tpc, lpt != 0);
                cudaEventRecord(e0, st);
                rs = launch_mixed_batch(sp.data(), sio.data(), order.data(), m, tpc, queue, status, st);
                if (rs != SSE_OK) break;
                cudaEventRecord(e1, st);
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    rs = cuda_fail(e, "autotune timing");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    ch = Choice{tpc, lpt};
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rs == SSE_OK) {
            std::lock_guard<std::mutex> lock(g_mu);
            g_cache[sig] = ch;
            save_choice(sig, ch);
        }
    }
    if (rs == SSE_OK) {
        std::vector<int> order = make_order(plans, slots_per_atom, n, ch.tpc, ch.lpt != 0);
        rs = launch_mixed_batch(plans, ios, order.data(), n, ch.tpc, queue, status, st);
    }
    if (!queue_in) cudaFreeAsync(queue, st);
    if (tpc_out) *tpc_out = ch.tpc;
    if (lpt_out) *lpt_out = ch.lpt;
    return rs;
}

bool batch_choice(Plan *const *plans, const sse_io *ios, int n, int *tpc, int *lpt) {
    if (n <= 0) return false;
    const unsigned long long sig = signature(plans, ios, n);
    std::lock_guard<std::mutex> lock(g_mu);
    load_cache_locked();
    auto it = g_cache.find(sig);
    if (it == g_cache.end()) return false;
    *tpc = it->second.tpc;
    *lpt = it->second.lpt;
    return true;
}

}  // namespace sse
