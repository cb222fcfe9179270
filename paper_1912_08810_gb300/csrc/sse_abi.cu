// C ABI of libsse_gb300.so: argument checks, plans, dispatch to the kernels.
// The operation and the readings of the paper it fixes are documented in include/sse.h.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "sse_internal.h"

namespace sse {

static thread_local std::string t_error;
static std::atomic<int32_t> g_inject{SSE_INJECT_NONE};

bool take_inject(int32_t kind) {
    int32_t expect = kind;
    return kind != SSE_INJECT_NONE && g_inject.compare_exchange_strong(expect, SSE_INJECT_NONE);
}

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_error = buf;
}

sse_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return SSE_E_CUDA;
}

double algorithmic_cmacs(const Dims &d, const std::vector<int32_t> &neigh) {
    int64_t bonds = 0;
    for (int32_t f : neigh) bonds += f >= 0;
    int64_t valid_w = 0;  // sum_w max(0, ne - |w + omega_first|): E and E - omega both on the grid
    for (int w = 0; w < d.nw; ++w) {
        const int64_t om = (int64_t)w + d.omega_first;
        const int64_t v = (int64_t)d.ne - (om < 0 ? -om : om);
        valid_w += v > 0 ? v : 0;
    }
    const double products = (double)bonds * d.nkz * d.ne * 12.0 * kNorb * kNorb * kNorb;  // M_ij once per (k', E')
    const double corr = (double)bonds * d.nkz * d.nqz * 9.0 * kBlk * (double)valid_w;      // sum over valid (q, w)
    return products + corr;
}

// True when `ptr` is memory a kernel of the current device can dereference.
static bool device_pointer(const void *ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static sse_status check_geometry(const sse_geometry *g) {
    if (!g) return set_error("geometry is NULL"), SSE_E_INVALID_ARG;
    if (g->nkz <= 0 || g->nqz <= 0 || g->ne <= 0 || g->nw <= 0 || g->na <= 0 || g->nb_max <= 0) {
        set_error("sizes must be positive (nkz=%d nqz=%d ne=%d nw=%d na=%d nb_max=%d)", g->nkz, g->nqz, g->ne,
                  g->nw, g->na, g->nb_max);
        return SSE_E_INVALID_ARG;
    }
    if (g->norb != kNorb) return set_error("norb must be 12 (got %d)", g->norb), SSE_E_INVALID_ARG;
    if (g->omega_first <= -(1 << 20) || g->omega_first >= (1 << 20))
        return set_error("omega_first out of range"), SSE_E_INVALID_ARG;
    if (g->dtype != SSE_C128 && g->dtype != SSE_C64) return set_error("unknown dtype %d", g->dtype), SSE_E_INVALID_ARG;
    if (g->mode != SSE_MODE_FP64 && g->mode != SSE_MODE_MIXED)
        return set_error("unknown mode %d", g->mode), SSE_E_INVALID_ARG;
    if ((int64_t)g->nkz * g->ne * g->na > (int64_t)1 << 40) return set_error("problem too large"), SSE_E_INVALID_ARG;
    if (!device_pointer(g->neigh)) return set_error("neigh is not a device pointer"), SSE_E_INVALID_ARG;
    if (!device_pointer(g->dH)) return set_error("dH is not a device pointer"), SSE_E_INVALID_ARG;
    return SSE_OK;
}

static sse_status check_io(const Plan &p, const sse_io *io) {
    if (!io) return set_error("io is NULL"), SSE_E_INVALID_ARG;
    if (!io->S_gt && !io->S_lt) return SSE_OK;
    if (io->S_gt && (!device_pointer(io->G_gt) || !device_pointer(io->D_gt) || !device_pointer(io->S_gt)))
        return set_error("G_gt, D_gt and S_gt must be device pointers"), SSE_E_INVALID_ARG;
    if (io->S_lt && (!device_pointer(io->G_lt) || !device_pointer(io->D_lt) || !device_pointer(io->S_lt)))
        return set_error("G_lt, D_lt and S_lt must be device pointers"), SSE_E_INVALID_ARG;
    (void)p;
    return SSE_OK;
}

}  // namespace sse

using namespace sse;

struct sse_plan_s : public Plan {
    std::vector<int32_t> neigh_host;
    double cmacs_per_sign = 0.0;
    double slots_per_atom = 0.0;  // mean valid neighbour slots per atom
};

namespace sse {
Plan *plan_core(sse_plan_t *p) { return p; }
double plan_slots_per_atom(const sse_plan_t *p) { return p->slots_per_atom; }
sse_status plan_check_io(sse_plan_t *p, const sse_io *io) { return check_io(*p, io); }
}  // namespace sse

namespace sse {
namespace {
void timing_accumulate(KernelTiming &t, int slot) {
    float a = 0.f, b = 0.f;
    if (cudaEventSynchronize(t.ev[slot][2]) == cudaSuccess && cudaEventElapsedTime(&a, t.ev[slot][0], t.ev[slot][1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, t.ev[slot][1], t.ev[slot][2]) == cudaSuccess) {
        t.prep_ms += a;
        t.main_ms += b;
    }
    cudaGetLastError();
    ++t.done;
}
void timing_free(KernelTiming &t) {
    for (auto &tr : t.ev)
        for (auto &e : tr)
            if (e) cudaEventDestroy(e), e = nullptr;
}
}  // namespace

int timing_slot(Plan &p) {
    KernelTiming &t = p.timing;
    if (!t.on) return -1;
    const int slot = (int)(t.issued % KernelTiming::kRing);
    if (t.issued - t.done >= KernelTiming::kRing) timing_accumulate(t, slot);
    ++t.issued;
    return slot;
}

void timing_mark(Plan &p, int slot, int which, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(p.timing.ev[slot][which], st);
}
}  // namespace sse

extern "C" {

int32_t sse_abi_version(void) { return 1; }

const char *sse_last_error(void) { return t_error.c_str(); }

const char *sse_status_string(sse_status s) {
    switch (s) {
        case SSE_OK: return "SSE_OK";
        case SSE_NOT_READY: return "SSE_NOT_READY";
        case SSE_E_INVALID_ARG: return "SSE_E_INVALID_ARG";
        case SSE_E_OUT_OF_MEMORY: return "SSE_E_OUT_OF_MEMORY";
        case SSE_E_CUDA: return "SSE_E_CUDA";
        case SSE_E_OVER_BUDGET: return "SSE_E_OVER_BUDGET";
        case SSE_E_TIMEOUT: return "SSE_E_TIMEOUT";
        case SSE_E_UNKNOWN_TICKET: return "SSE_E_UNKNOWN_TICKET";
        case SSE_E_SHUTDOWN: return "SSE_E_SHUTDOWN";
        case SSE_E_CANCELLED: return "SSE_E_CANCELLED";
        case SSE_E_BOUNDS: return "SSE_E_BOUNDS";
        default: return "SSE_E_UNKNOWN_STATUS";
    }
}

sse_status sse_plan(const sse_geometry *geo, sse_plan_t **out) {
    if (!out) return set_error("out is NULL"), SSE_E_INVALID_ARG;
    *out = nullptr;
    sse_status st = check_geometry(geo);
    if (st != SSE_OK) return st;
    sse_plan_s *p = new (std::nothrow) sse_plan_s();
    if (!p) return set_error("host allocation failed"), SSE_E_OUT_OF_MEMORY;
    p->geo = *geo;
    p->d = Dims{geo->nkz, geo->nqz, geo->ne, geo->nw, geo->na, geo->nb_max, geo->omega_first};
    cudaGetDevice(&p->device);
    const size_t nn = (size_t)geo->na * geo->nb_max;
    try {
        p->neigh_host.resize(nn);
    } catch (...) {
        delete p;
        return set_error("host allocation failed"), SSE_E_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaMemcpy(p->neigh_host.data(), geo->neigh, nn * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "copy neigh to host");
    }
    for (size_t i = 0; i < nn; ++i) {
        const int32_t f = p->neigh_host[i];
        if (f < -1 || f >= geo->na) {
            set_error("neigh[%zu][%zu] = %d is outside [-1, %d)", i / geo->nb_max, i % geo->nb_max, f, geo->na);
            delete p;
            return SSE_E_INVALID_ARG;
        }
    }
    p->cmacs_per_sign = algorithmic_cmacs(p->d, p->neigh_host);
    // reverse bonds (for the phonon pre-combination of Eq. 3)
    std::vector<int32_t> rev(nn, -1);
    p->rev_ok = true;
    for (int a = 0; a < geo->na; ++a)
        for (int s = 0; s < geo->nb_max; ++s) {
            const int32_t b = p->neigh_host[(size_t)a * geo->nb_max + s];
            if (b < 0) continue;
            for (int s2 = 0; s2 < geo->nb_max && rev[(size_t)a * geo->nb_max + s] < 0; ++s2)
                if (p->neigh_host[(size_t)b * geo->nb_max + s2] == a) rev[(size_t)a * geo->nb_max + s] = s2;
            if (rev[(size_t)a * geo->nb_max + s] < 0) p->rev_ok = false;
        }
    {
        size_t valid = 0;
        for (int32_t f : p->neigh_host) valid += f >= 0;
        p->slots_per_atom = (double)valid / geo->na;
    }
    e = cudaMalloc(&p->d_status, sizeof(int32_t));
    if (e == cudaSuccess) {
        e = cudaMalloc(&p->d_rev, nn * sizeof(int32_t));
        if (e != cudaSuccess) cudaFree(p->d_status);
    }
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorMemoryAllocation ? (set_error("cudaMalloc of the plan's small tables"), SSE_E_OUT_OF_MEMORY)
                                              : cuda_fail(e, "cudaMalloc of the plan's small tables");
    }
    cudaMemset(p->d_status, 0, sizeof(int32_t));
    cudaMemcpy(p->d_rev, rev.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice);
    p->workspace_bytes = sizeof(int32_t) + (int64_t)(nn * sizeof(int32_t));
    if (geo->mode == SSE_MODE_MIXED) {
        p->kernel_id = 1;
        st = mixed_plan_init(*p);
        if (st != SSE_OK) {
            mixed_plan_free(*p);
            cudaFree(p->d_status);
            cudaFree(p->d_rev);
            delete p;
            return st;
        }
    } else {
        p->kernel_id = 0;
        p->tile_e = 1;
    }
    *out = p;
    return SSE_OK;
}

sse_status sse_plan_destroy(sse_plan_t *plan) {
    if (!plan) return SSE_OK;
    if (plan->last_stream) cudaStreamSynchronize(plan->last_stream);
    mixed_plan_free(*plan);
    timing_free(plan->timing);
    if (plan->d_status) cudaFree(plan->d_status);
    if (plan->d_rev) cudaFree(plan->d_rev);
    if (plan->dt_scratch) cudaFree(plan->dt_scratch);
    if (plan->staging) cudaFree(plan->staging);
    if (plan->side) {
        cudaStreamSynchronize(plan->side);
        cudaStreamDestroy(plan->side);
    }
    for (cudaEvent_t e : plan->ev_order)
        if (e) cudaEventDestroy(e);
    delete plan;
    return SSE_OK;
}

sse_status sse_plan_query(const sse_plan_t *plan, sse_plan_info *info) {
    if (!plan || !info) return set_error("plan or info is NULL"), SSE_E_INVALID_ARG;
    const Dims &d = plan->d;
    const double eb = (double)elem_bytes(plan->geo.dtype);
    info->mode = plan->geo.mode;
    info->dtype = plan->geo.dtype;
    info->points = (int64_t)d.nkz * d.ne * d.na;
    info->flops_per_sign = 8.0 * plan->cmacs_per_sign;
    info->bytes_per_sign = eb * (2.0 * g_elems(d) + d_elems(d) + 0.5 * dh_elems(d)) + 0.5 * 4.0 * d.na * d.nb;
    info->workspace_bytes = plan->workspace_bytes + (int64_t)plan->staging_bytes + (int64_t)plan->dt_scratch_bytes;
    info->tile_e = plan->tile_e;
    info->kernel_id = plan->kernel_id;
    return SSE_OK;
}


static sse_status dispatch(sse_plan_t *plan, const sse_io &io, cudaStream_t st) {
    plan->last_stream = st;
    if (plan->kernel_id == 1) return launch_mixed(*plan, io, st);
    const int ts = timing_slot(*plan);
    timing_mark(*plan, ts, 0, st);
    timing_mark(*plan, ts, 1, st);
    const sse_status rs = launch_fp64_direct(*plan, io, st);
    timing_mark(*plan, ts, 2, st);
    return rs;
}

sse_status sse_execute(sse_plan_t *plan, const sse_io *io, void *stream) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    sse_status st = check_io(*plan, io);
    if (st != SSE_OK) return st;
    return dispatch(plan, *io, (cudaStream_t)stream);
}

sse_status sse_dtilde(const sse_plan_t *plan, const void *D, void *Dt, void *stream) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    if (!device_pointer(D) || !device_pointer(Dt)) return set_error("D and Dt must be device pointers"), SSE_E_INVALID_ARG;
    return launch_dtilde(*plan, D, Dt, (cudaStream_t)stream);
}

sse_status sse_retarded(const sse_plan_t *plan, const void *S_gt, const void *S_lt, void *S_r, void *stream) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    if (!device_pointer(S_gt) || !device_pointer(S_lt) || !device_pointer(S_r))
        return set_error("S_gt, S_lt and S_r must be device pointers"), SSE_E_INVALID_ARG;
    return launch_retarded(*plan, S_gt, S_lt, S_r, (cudaStream_t)stream);
}

sse_status sse_pi(sse_plan_t *plan, const void *G_gt, const void *G_lt, void *Pi_gt, void *Pi_lt, void *stream) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    if (!Pi_gt && !Pi_lt) return SSE_OK;
    if (!device_pointer(G_gt) || !device_pointer(G_lt))
        return set_error("G_gt and G_lt must both be device pointers (each sign of Pi pairs one with the other)"),
               SSE_E_INVALID_ARG;
    if ((Pi_gt && !device_pointer(Pi_gt)) || (Pi_lt && !device_pointer(Pi_lt)))
        return set_error("Pi_gt / Pi_lt must be device pointers"), SSE_E_INVALID_ARG;
    plan->last_stream = (cudaStream_t)stream;
    return launch_pi(*plan, G_gt, G_lt, Pi_gt, Pi_lt, (cudaStream_t)stream);
}

sse_status sse_execute_full(sse_plan_t *plan, const sse_io *io, void *S_r, void *stream) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    sse_status rs = check_io(*plan, io);
    if (rs != SSE_OK) return rs;
    if (!plan->rev_ok) {
        set_error("the pre-combination needs every bond's reverse: some neigh[a][slot] = b has no slot of b holding a");
        return SSE_E_INVALID_ARG;
    }
    if (S_r && (!io->S_gt || !io->S_lt)) return set_error("Sigma^R needs both signs"), SSE_E_INVALID_ARG;
    if (S_r && !device_pointer(S_r)) return set_error("S_r must be a device pointer"), SSE_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    plan->last_stream = st;
    if (plan->kernel_id == 1) {
        rs = launch_mixed(*plan, *io, st, /*dfull=*/true);
    } else {
        // the FP64 form reads Dt in its innermost loop: pre-combine into plan-owned scratch
        const size_t db = d_elems(plan->d) * elem_bytes(plan->geo.dtype);
        if (plan->dt_scratch_bytes < 2 * db) {
            if (plan->dt_scratch) cudaFree(plan->dt_scratch);
            plan->dt_scratch = nullptr;
            plan->dt_scratch_bytes = 0;
            cudaError_t e = take_inject(SSE_INJECT_ALLOC_FAIL) ? cudaErrorMemoryAllocation : cudaMalloc(&plan->dt_scratch, 2 * db);
            if (e != cudaSuccess) {
                cudaGetLastError();
                plan->dt_scratch = nullptr;
                return set_error("cudaMalloc of %zu bytes for Dt failed", 2 * db), SSE_E_OUT_OF_MEMORY;
            }
            plan->dt_scratch_bytes = 2 * db;
        }
        sse_io dio = *io;
        if (io->S_gt) {
            rs = launch_dtilde(*plan, io->D_gt, plan->dt_scratch, st);
            dio.D_gt = plan->dt_scratch;
        }
        if (rs == SSE_OK && io->S_lt) {
            rs = launch_dtilde(*plan, io->D_lt, (char *)plan->dt_scratch + db, st);
            dio.D_lt = (char *)plan->dt_scratch + db;
        }
        if (rs == SSE_OK) rs = dispatch(plan, dio, st);
    }
    if (rs == SSE_OK && S_r) rs = launch_retarded(*plan, io->S_gt, io->S_lt, S_r, st);
    return rs;
}

sse_status sse_execute_host(sse_plan_t *plan, const sse_io *h, void *stream) {
    if (!plan || !h) return set_error("plan or io is NULL"), SSE_E_INVALID_ARG;
    const Dims &d = plan->d;
    const size_t eb = elem_bytes(plan->geo.dtype);
    const size_t gb = g_elems(d) * eb, db = d_elems(d) * eb;
    const bool sgn[2] = {h->S_gt != nullptr, h->S_lt != nullptr};
    const void *hg[2] = {h->G_gt, h->G_lt}, *hd[2] = {h->D_gt, h->D_lt};
    void *hs[2] = {h->S_gt, h->S_lt};
    for (int s = 0; s < 2; ++s)
        if (sgn[s] && (!hg[s] || !hd[s])) return set_error("missing host input for a requested sign"), SSE_E_INVALID_ARG;
    const size_t need = 2 * (2 * gb + db);  // per sign: G, Dt, Sigma
    if (plan->staging_bytes < need) {
        if (plan->staging) cudaFree(plan->staging);
        plan->staging = nullptr;
        plan->staging_bytes = 0;
        cudaError_t e = cudaMalloc(&plan->staging, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error("cudaMalloc of %zu staging bytes failed", need), SSE_E_OUT_OF_MEMORY;
        }
        plan->staging_bytes = need;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)plan->staging;
    auto fail = [&](cudaError_t e, const char *what) {
        cudaStreamSynchronize(st);
        if (plan->side) cudaStreamSynchronize(plan->side);
        plan->last_stream = st;
        return cuda_fail(e, what);
    };
    // one sign: copies in, kernels, copies out on the caller's stream.  Both signs: sign 0
    // on the caller's stream, sign 1 on the plan's side stream, its input copies after sign
    // 0's (full link bandwidth for the first kernels' inputs), its kernels after sign 0's
    // (executions of a plan do not overlap), so that sign 1's inputs and sign 0's Sigma
    // move while the other sign computes
    const bool both = sgn[0] && sgn[1];
    if (both && !plan->side) {
        cudaError_t e = cudaStreamCreateWithFlags(&plan->side, cudaStreamNonBlocking);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            if (!plan->ev_order[k]) e = cudaEventCreateWithFlags(&plan->ev_order[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "create the second stream of sse_execute_host");
    }
    for (int s = 0; s < 2; ++s) {
        if (!sgn[s]) continue;
        cudaStream_t ss = (both && s == 1) ? plan->side : st;
        char *g = base + s * (2 * gb + db), *dt = g + gb, *sg = dt + db;
        cudaError_t e = cudaSuccess;
        if (both && s == 1) e = cudaStreamWaitEvent(ss, plan->ev_order[0], 0);  // after sign 0's inputs
        if (e == cudaSuccess) e = cudaMemcpyAsync(g, hg[s], gb, cudaMemcpyHostToDevice, ss);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dt, hd[s], db, cudaMemcpyHostToDevice, ss);
        if (e == cudaSuccess && both && s == 0) e = cudaEventRecord(plan->ev_order[0], ss);
        if (e == cudaSuccess && both && s == 1) e = cudaStreamWaitEvent(ss, plan->ev_order[1], 0);  // after sign 0's kernels
        if (e != cudaSuccess) return fail(e, "copy inputs to the device");
        sse_io dio{};
        if (s == 0) {
            dio.G_gt = g;
            dio.D_gt = dt;
            dio.S_gt = sg;
        } else {
            dio.G_lt = g;
            dio.D_lt = dt;
            dio.S_lt = sg;
        }
        const sse_status rs = dispatch(plan, dio, ss);
        if (rs != SSE_OK) {
            cudaStreamSynchronize(st);
            if (plan->side) cudaStreamSynchronize(plan->side);
            plan->last_stream = st;
            return rs;
        }
        if (both && s == 0) e = cudaEventRecord(plan->ev_order[1], ss);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs[s], sg, gb, cudaMemcpyDeviceToHost, ss);
        if (e != cudaSuccess) return fail(e, "copy Sigma to the host");
    }
    cudaError_t e = cudaSuccess;
    if (both) {
        e = cudaEventRecord(plan->ev_order[2], plan->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, plan->ev_order[2], 0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    plan->last_stream = st;
    if (e != cudaSuccess) return fail(e, "synchronise after sse_execute_host");
    return SSE_OK;
}

// Shared checks of a batch: every plan mixed-mode with the same Nkz, Nw, omega_first, dtype.
static sse_status check_batch(sse_plan_t *const *plans, const sse_io *ios, int32_t n) {
    if (n < 0 || (n > 0 && (!plans || !ios))) return set_error("bad batch arguments"), SSE_E_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i) {
        if (!plans[i]) return set_error("plans[%d] is NULL", i), SSE_E_INVALID_ARG;
        if (plans[i]->kernel_id != 1) return set_error("plans[%d] is not a mixed-mode plan", i), SSE_E_INVALID_ARG;
        const Dims &a = plans[i]->d, &b = plans[0]->d;
        if (a.nkz != b.nkz || a.nw != b.nw || a.omega_first != b.omega_first ||
            plans[i]->geo.dtype != plans[0]->geo.dtype)
            return set_error("plans[%d] differs from plans[0] in nkz, nw, omega_first or dtype", i), SSE_E_INVALID_ARG;
        sse_status st = check_io(*plans[i], &ios[i]);
        if (st != SSE_OK) return st;
    }
    return SSE_OK;
}

sse_status sse_execute_batch(sse_plan_t *const *plans, const sse_io *ios, int32_t n, void *stream) {
    sse_status st = check_batch(plans, ios, n);
    if (st != SSE_OK || n == 0) return st;
    std::vector<Plan *> ps((size_t)n);
    std::vector<double> slots((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        ps[i] = plans[i];
        slots[i] = plans[i]->slots_per_atom;
        plans[i]->last_stream = (cudaStream_t)stream;
    }
    return run_batch(ps.data(), slots.data(), ios, n, (cudaStream_t)stream, plans[0]->d_status, nullptr, nullptr);
}

sse_status sse_batch_tuning(sse_plan_t *const *plans, const sse_io *ios, int32_t n, int32_t *tiles_per_unit,
                            int32_t *longest_first) {
    sse_status st = check_batch(plans, ios, n);
    if (st != SSE_OK) return st;
    if (!tiles_per_unit || !longest_first) return set_error("output pointers are NULL"), SSE_E_INVALID_ARG;
    std::vector<Plan *> ps((size_t)n);
    for (int32_t i = 0; i < n; ++i) ps[i] = plans[i];
    int tpc = 0, lpt = 0;
    if (!batch_choice(ps.data(), ios, n, &tpc, &lpt)) return SSE_NOT_READY;
    *tiles_per_unit = tpc;
    *longest_first = lpt;
    return SSE_OK;
}

sse_status sse_plan_set_timing(sse_plan_t *plan, int32_t enable) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    KernelTiming &t = plan->timing;
    if (enable) {
        for (auto &tr : t.ev)
            for (auto &e : tr)
                if (!e) {
                    cudaError_t err = cudaEventCreate(&e);
                    if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate(timing)");
                }
    }
    t.on = enable != 0;
    t.issued = t.done = 0;
    t.prep_ms = t.main_ms = 0.0;
    return SSE_OK;
}

sse_status sse_plan_timing(sse_plan_t *plan, double *prep_ms, double *main_ms, int64_t *calls) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    KernelTiming &t = plan->timing;
    while (t.done < t.issued) timing_accumulate(t, (int)(t.done % KernelTiming::kRing));
    if (prep_ms) *prep_ms = t.prep_ms;
    if (main_ms) *main_ms = t.main_ms;
    if (calls) *calls = t.done;
    return SSE_OK;
}

sse_status sse_debug_inject(int32_t kind) {
    if (kind != SSE_INJECT_NONE && kind != SSE_INJECT_STALL && kind != SSE_INJECT_ALLOC_FAIL)
        return set_error("unknown injection kind %d", kind), SSE_E_INVALID_ARG;
    g_inject.store(kind);
    return SSE_OK;
}

sse_status sse_plan_status(sse_plan_t *plan) {
    if (!plan) return set_error("plan is NULL"), SSE_E_INVALID_ARG;
    cudaError_t e = plan->last_stream ? cudaStreamSynchronize(plan->last_stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise plan stream");
    int32_t v = 0;
    e = cudaMemcpy(&v, plan->d_status, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read plan status");
    if (v != 0) {
        cudaMemset(plan->d_status, 0, sizeof v);
        if (v & kStatusBounds) {
            set_error("a kernel of this plan computed an index outside one of its buffers (status %d)", v);
            return SSE_E_BOUNDS;
        }
        set_error("a device-side wait of this plan expired (code %d)", v);
        return SSE_E_TIMEOUT;
    }
    return SSE_OK;
}

}  // extern "C"
