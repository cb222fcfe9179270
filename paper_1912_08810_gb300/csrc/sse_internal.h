// Internal declarations shared by the translation units of libsse_gb300.so.
// Nothing here is part of the C ABI (include/sse.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sse.h"

namespace sse {

// Bounds-checked build (compiled with -DSSE_BOUNDS_CHECK into a library of its own): each
// global index a kernel computes is checked against the extent of its buffer; a violation
// sets kStatusBounds in the status word (read by sse_plan_status as SSE_E_BOUNDS) and the
// access is skipped.  Nothing traps.  In the normal build the checks compile away.
constexpr int32_t kStatusTimeout = 1, kStatusBounds = 2;
#ifdef SSE_BOUNDS_CHECK
__device__ __forceinline__ bool bc_in(long long idx, long long n, int32_t *status) {
    const bool ok = idx >= 0 && idx < n;
    if (!ok && status) atomicOr(status, kStatusBounds);
    return ok;
}
#define SSE_BC(idx, n, status) ::sse::bc_in((long long)(idx), (long long)(n), (status))
#else
#define SSE_BC(idx, n, status) true
#endif

constexpr int kNorb = 12;             // orbitals per atom (the only size the kernels take)
constexpr int kBlk = kNorb * kNorb;   // complex values per norb x norb block
constexpr int kN3D = 3;               // vibration directions i, j

// Sizes of one instance (Table 1 symbols) in the form the kernels take.
struct Dims {
    int32_t nkz, nqz, ne, nw, na, nb, omega_first;
};

// Event timing of sse_execute (sse_plan_set_timing): a ring of (start, after the workspace
// pass, after the main kernel) event triples, accumulated when a slot is reused or on query.
struct KernelTiming {
    static constexpr int kRing = 64;
    bool on = false;
    cudaEvent_t ev[kRing][3] = {};
    int64_t issued = 0, done = 0;
    double prep_ms = 0.0, main_ms = 0.0;
};

struct Plan {
    sse_geometry geo{};
    Dims d{};
    int device = 0;
    int kernel_id = 0;
    int tile_e = 1;
    int32_t *d_status = nullptr;      // device status word written by kernels with bounded waits
    void *staging = nullptr;          // device staging of sse_execute_host
    size_t staging_bytes = 0;
    // sse_execute_host with both signs: a second (non-blocking) stream carries the second
    // sign, so that its copies overlap the first sign's kernels; events order the two
    cudaStream_t side = nullptr;
    cudaEvent_t ev_order[3] = {};     // caller stream: inputs of sign 0 copied, sign 0 computed; side stream: done
    cudaStream_t last_stream = nullptr;
    int64_t workspace_bytes = 0;
    // Mixed-path workspace (see sse_mixed.cu), Nkz = 5 tensor-core form: per sign, G
    // re-encoded as bf16 hi/lo slices in operand layout ((ne * na + 1) slices, the last zero),
    // then the slot tables of every (atom, slot)
    void *mixed_ws = nullptr;
    size_t mixed_ws_bytes = 0;
    // Reverse bonds for the phonon pre-combination (Eq. 3): rev[a][slot] = the first slot s'
    // of b = neigh[a][slot] with neigh[b][s'] = a; -1 for an empty slot or a bond whose
    // reverse is not listed (rev_ok is then false).
    int32_t *d_rev = nullptr;
    bool rev_ok = false;
    // Dt of both signs for the FP64 form of sse_execute_full (allocated on first use)
    void *dt_scratch = nullptr;
    size_t dt_scratch_bytes = 0;
    KernelTiming timing;
};

// Timing hooks: timing_slot returns the ring slot of this call (-1 when timing is off);
// timing_mark records event `which` (0 start, 1 after the workspace pass, 2 end) on `st`.
int timing_slot(Plan &p);
void timing_mark(Plan &p, int slot, int which, cudaStream_t st);

// Thread-local error message for sse_last_error().
void set_error(const char *fmt, ...);
sse_status cuda_fail(cudaError_t e, const char *what);

inline size_t elem_bytes(int dtype) { return dtype == SSE_C128 ? 16 : 8; }
inline size_t g_elems(const Dims &d) { return (size_t)d.nkz * d.ne * d.na * kBlk; }
inline size_t d_elems(const Dims &d) { return (size_t)d.nqz * d.nw * d.na * d.nb * kN3D * kN3D; }
inline size_t dh_elems(const Dims &d) { return (size_t)d.na * d.nb * kN3D * kBlk; }

// Algorithmic work per sign (complex MACs): the q/w-independent products once per
// (k', E', a, slot) plus the correlation over the valid (q, w).
double algorithmic_cmacs(const Dims &d, const std::vector<int32_t> &neigh_host);

// Kernel launchers (return SSE_OK or an error after set_error).
sse_status launch_fp64_direct(const Plan &p, const sse_io &io, cudaStream_t st);
// dfull: io.D_gt / io.D_lt hold the full phonon tensors [nqz][nw][na][nb+1][3][3]; the
// kernels then form Dt = D_ba - D_bb - D_aa + D_ab where they read it (needs p.rev_ok).
sse_status launch_mixed(Plan &p, const sse_io &io, cudaStream_t st, bool dfull = false);
// The steps on either side (sse_edges.cu): Dt of one sign into `dt`, Sigma^R from both signs.
sse_status launch_dtilde(const Plan &p, const void *D, void *dt, cudaStream_t st);
sse_status launch_retarded(const Plan &p, const void *S_gt, const void *S_lt, void *S_r, cudaStream_t st);
// The phonon self-energy of Eqs. 4-5 (sse_pi.cu), FP64.
sse_status launch_pi(const Plan &p, const void *G_gt, const void *G_lt, void *Pi_gt, void *Pi_lt, cudaStream_t st);
// Persistent launch over n instances in the given order (all plans mixed, with equal
// nkz, nw, omega_first and dtype), `tpc` tiles per work unit, `queue` a device counter;
// expired device waits are recorded in the device word `status`.
sse_status launch_mixed_batch(Plan *const *plans, const sse_io *ios, const int *order, int n, int tpc,
                              int32_t *queue, int32_t *status, cudaStream_t st);
// Batched execution with the autotuned work split (sse_batch.cu); slots_per_atom[i] is the
// mean number of valid neighbour slots of plans[i]; `status` receives expired device waits.
// Without allow_tune an untuned shape runs with the default split instead of tuning.  With
// `queue` (a device int32 owned by the caller) no work counter is allocated.
sse_status run_batch(Plan *const *plans, const double *slots_per_atom, const sse_io *ios, int n, cudaStream_t st,
                     int32_t *status, int *tpc_out, int *lpt_out, bool allow_tune = true, int32_t *queue = nullptr);

// One-shot test hooks (sse_debug_inject): take_inject(kind) returns true once after the
// hook was armed with that kind.
bool take_inject(int32_t kind);
bool batch_choice(Plan *const *plans, const sse_io *ios, int n, int *tpc, int *lpt);
sse_status mixed_plan_init(Plan &p);
void mixed_plan_free(Plan &p);

}  // namespace sse
