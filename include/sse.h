/*
 * sse.h -- C ABI of the GB300 scattering self-energy library (libsse_gb300.so).
 *
 * The library evaluates the electron scattering self-energy of Eq. 3 (Section 2),
 * after the pre-combination of the phonon Green's function described in Section 3
 * ("Dataflow Optimizations", inputs list):
 *
 *   Sigma^s[k,E,a] = sum_{slot: f = neigh[a,slot] >= 0} sum_{i,j in x,y,z} sum_{q < nqz}
 *                    sum_{w < nw, E' = E - (w + omega_first) >= 0}
 *                    Dt^s[q,w,a,slot,i,j] * dH[a,slot,i] . G^s[(k-q) mod nkz, E', f] . dH[a,slot,j]^dagger
 *
 * for both signs s in {>, <}, on norb x norb complex blocks (norb = 12).  Readings of
 * the paper fixed by this ABI:
 *   - the prefactor i and the frequency weight of Eq. 3 are the caller's (factor 1);
 *   - the sum index l of Eq. 3 is the neighbour slot;
 *   - grad_j H_ba is the conjugate transpose of the stored dH[a,slot,j];
 *   - kz - qz wraps modulo nkz; E - omega off the energy grid contributes 0;
 *   - Sigma is overwritten, not accumulated.
 *
 * Layouts (row-major; complex = interleaved re/im, double2 for SSE_C128, float2 for
 * SSE_C64; every array of one plan uses the plan's dtype):
 *   G^s   [nkz][ne][na][12][12]       device, read-only
 *   Dt^s  [nqz][nw][na][nb_max][3][3] device, read-only
 *   dH    [na][nb_max][3][12][12]     device, read-only, borrowed by the plan
 *   neigh [na][nb_max] int32          device, read-only, borrowed by the plan; -1 = empty slot
 *   Sigma [nkz][ne][na][12][12]       device, written
 *
 * Ownership: the caller owns every buffer.  A plan borrows neigh and dH for its whole
 * lifetime (they must not change after sse_plan; the neighbour list is validated
 * once, at sse_plan).  A server ticket borrows its sse_io buffers until sse_poll
 * returns a final status.  The library owns only its plans, their workspace and the
 * server's queues.
 *
 * Errors: every entry point returns an sse_status; no C++ exception crosses the ABI,
 * nothing aborts and no kernel traps.  sse_last_error() gives the calling thread's
 * message for the last failure.  Kernels that wait on the device stop after a bounded
 * time and record SSE_E_TIMEOUT in the plan's device status (see sse_plan_status).
 *
 * Streams are passed as `void *` holding a cudaStream_t (NULL = legacy default stream).
 */
#ifndef SSE_GB300_SSE_H
#define SSE_GB300_SSE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SSE_API __attribute__((visibility("default")))
#else
#define SSE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sse_status;
enum {
    SSE_OK = 0,
    SSE_NOT_READY = 1,          /* sse_poll: the request is still queued or running */
    SSE_E_INVALID_ARG = -1,     /* bad pointer, size, dtype, mode or neighbour index */
    SSE_E_OUT_OF_MEMORY = -2,   /* a device or host allocation failed */
    SSE_E_CUDA = -3,            /* a CUDA runtime call failed (message has the CUDA error) */
    SSE_E_OVER_BUDGET = -4,     /* the request can never fit the server's memory budget */
    SSE_E_TIMEOUT = -5,         /* a bounded device or host wait expired */
    SSE_E_UNKNOWN_TICKET = -6,  /* sse_poll: no such ticket (or already collected) */
    SSE_E_SHUTDOWN = -7,        /* the server is shutting down or was destroyed */
    SSE_E_CANCELLED = -9,       /* the request was cancelled before it ran */
    SSE_E_BOUNDS = -10          /* bounds-checked build only: a kernel computed an index outside a buffer */
};

typedef enum { SSE_C128 = 0, SSE_C64 = 1 } sse_dtype;

/* SSE_MODE_FP64: every product and sum in FP64 (the oracle-matching reference form).
 * SSE_MODE_MIXED: products on the tensor cores from split-bf16 operands with FP32
 * accumulation; the sum over neighbour slots into Sigma is FP64 for SSE_C128 and kept in
 * the output's own FP32 for SSE_C64. */
typedef enum { SSE_MODE_FP64 = 0, SSE_MODE_MIXED = 1 } sse_mode;

typedef struct {
    int32_t nkz, nqz, ne, nw, na, nb_max;
    int32_t norb;         /* must be 12 */
    int32_t omega_first;  /* w means (w + omega_first) energy-grid steps; may be negative: a grid
                             spanning both signs gives the two-sided exchange E -+ hbar omega */
    const int32_t *neigh; /* device [na][nb_max] */
    const void *dH;       /* device [na][nb_max][3][12][12] */
    int32_t dtype;        /* sse_dtype */
    int32_t mode;         /* sse_mode */
} sse_geometry;

typedef struct {
    const void *G_gt, *G_lt; /* device G^>, G^< */
    const void *D_gt, *D_lt; /* device Dt^>, Dt^< */
    void *S_gt, *S_lt;       /* device Sigma^>, Sigma^<; NULL skips that sign */
} sse_io;

typedef struct sse_plan_s sse_plan_t;
typedef struct sse_server_s sse_server_t;

typedef struct {
    int32_t mode, dtype;
    int64_t points;          /* nkz * ne * na output blocks per sign */
    double flops_per_sign;   /* algorithmic real flops per sign (8 per complex MAC) */
    double bytes_per_sign;   /* algorithmic HBM bytes per sign: read G, Dt, dH once, write Sigma */
    int64_t workspace_bytes; /* device memory owned by the plan */
    int32_t tile_e;          /* energies per tile of the chosen kernel */
    int32_t kernel_id;       /* 0 = FP64 direct, 1 = mixed tensor-core */
} sse_plan_info;

/* Validate the geometry (copies neigh to the host once to range-check it: every entry
 * in [-1, na)), choose the kernel and its tiles, and allocate the plan.  On success
 * *out owns a plan that the caller frees with sse_plan_destroy.  A mixed-mode plan with
 * nkz = 5 and nw <= 50 (the warp-specialised tensor-core form) also owns a workspace of
 * 2 (ne na + 1) x 8 KB (G re-encoded for the tensor-core product dH_i G) plus
 * 2 na nb x (2 KB (nw + 14) + 26 KB) (each bond's operand tables), one half per sign:
 * 2.6 GB for nkz = 5, ne = 256, na = 512, nb = 4, nw = 32.  Its size is reported in
 * sse_plan_info.workspace_bytes.  Executions of one plan must not overlap on the GPU:
 * issue them on one stream or order them with events.  The batched form and the server
 * keep to this on their own (a plan that appears twice in one batch falls back to the
 * form without workspace; a server round holds a plan once). */
SSE_API sse_status sse_plan(const sse_geometry *geo, sse_plan_t **out);
SSE_API sse_status sse_plan_destroy(sse_plan_t *plan);
SSE_API sse_status sse_plan_query(const sse_plan_t *plan, sse_plan_info *info);

/* Enqueue Sigma^> and/or Sigma^< for one instance on `stream` (asynchronous, stream
 * ordered).  io buffers must follow the plan's geometry and dtype. */
SSE_API sse_status sse_execute(sse_plan_t *plan, const sse_io *io, void *stream);

/* ---- the steps on either side of Sigma -----------------------------------------------------
 *
 * The full phonon tensor D^s of Section 2 is [nqz][nw][na][nb_max + 1][3][3]: block slot
 * (< nb_max) of atom a couples a to b = neigh[a][slot] (D_ab), block nb_max is the diagonal
 * D_aa.  Eq. 3 uses the pre-combination (Section 3, "Dataflow Optimizations", input list)
 *   Dt[q][w][a][slot] = D_ba - D_bb - D_aa + D_ab,
 * where D_ba is the block of b at the first slot s' with neigh[b][s'] = a.  A plan whose
 * neighbour list has a bond without its reverse cannot form it (SSE_E_INVALID_ARG).  Dt is
 * summed in FP64 in the order ((D_ba - D_bb) - D_aa) + D_ab and rounded once to the plan's
 * dtype; an empty slot gives 0. */

/* Pre-combine one sign: D device [nqz][nw][na][nb_max + 1][3][3] -> Dt device
 * [nqz][nw][na][nb_max][3][3], both in the plan's dtype.  Asynchronous on `stream`. */
SSE_API sse_status sse_dtilde(const sse_plan_t *plan, const void *D, void *Dt, void *stream);

/* The retarded component (Section 2, the relation after Eq. 5): S_r = (S_gt - S_lt) / 2,
 * elementwise over the plan's Sigma shape [nkz][ne][na][12][12].  Asynchronous. */
SSE_API sse_status sse_retarded(const sse_plan_t *plan, const void *S_gt, const void *S_lt, void *S_r, void *stream);

/* The chain from the phonon Green's function to Sigma^R on `stream`: io->D_gt / io->D_lt hold
 * the FULL phonon tensors [nqz][nw][na][nb_max + 1][3][3]; Sigma^> and Sigma^< are written as
 * by sse_execute, and Sigma^R as well when S_r is not NULL (both signs needed then).  The
 * mixed form pre-combines Dt where its kernels read it (the tensor is never stored; results
 * equal sse_dtilde followed by sse_execute bit for bit); the FP64 form pre-combines into
 * plan-owned scratch (2 x the Dt size, allocated on first use, reported in workspace_bytes). */
SSE_API sse_status sse_execute_full(sse_plan_t *plan, const sse_io *io, void *S_r, void *stream);

/* ---- the phonon self-energy ----------------------------------------------------------------
 *
 * Pi^> and/or Pi^< of Eq. 5 (the N_B off-diagonal blocks, Section 2 keeps these) and Eq. 4
 * (the diagonal block), on the plan's geometry:
 *   Pi^s[q][w][a][slot][i][j] = sum_k sum_{E : E' = E + (w + omega_first) < ne}
 *       tr{ dH[a][slot][i]^dagger . G^s[(k + q) mod nkz][E'][a] . dH[a][slot][j] . G^s'[k][E][b] }
 * for b = neigh[a][slot] >= 0 (zero block for an empty slot), s' the opposite sign of s, and
 *   Pi^s[q][w][a][nb_max][i][j] = - sum over the atom's non-empty slots of the above.
 * Readings: the prefactors -i (Eq. 4) and +i (Eq. 5) and the weight dE/2pi are the caller's,
 * their relative sign kept (the diagonal block is minus the sum); Eq. 4's index l is the
 * neighbour; grad_i H_ba = dH[a][slot][i]^dagger; kz + qz wraps modulo nkz; E + omega above
 * the energy grid contributes nothing.  Layout: Pi [nqz][nw][na][nb_max + 1][3][3] in the plan's
 * dtype (the shape of the full phonon Green's function).  Both G^> and G^< are read for either
 * sign.  FP64 arithmetic on the FP64 pipe, whatever the plan's mode; nw <= 90.  Asynchronous
 * on `stream`; a NULL Pi pointer skips that sign. */
SSE_API sse_status sse_pi(sse_plan_t *plan, const void *G_gt, const void *G_lt, void *Pi_gt, void *Pi_lt, void *stream);

/* Same computation with HOST buffers (pageable or pinned): copies the inputs to
 * plan-owned device staging on `stream`, runs, copies Sigma back and synchronises
 * the stream before returning.  Staging is allocated on first use and kept.  With both
 * signs requested, the second sign runs on a plan-owned second stream (created on first
 * use) whose input copies follow the first sign's and whose kernels follow the first
 * sign's kernels, so that with pinned host buffers the copies of one sign overlap the
 * other's computation; the call returns after both. */
SSE_API sse_status sse_execute_host(sse_plan_t *plan, const sse_io *host_io, void *stream);

/* Batched form: evaluate n independent instances -- each with its own plan and
 * buffers, uneven na, ne, nb_max and nqz allowed -- in one persistent launch of the
 * mixed kernel: one CTA per SM pulls work units (sign, atom, range of energy tiles) from
 * a device counter until none are left.  All plans must be SSE_MODE_MIXED with equal
 * nkz, nw, omega_first and dtype.  The split of the work (tiles per unit, and whether the
 * longest units enter the queue first) comes from an exhaustive autotuner: the first call
 * for a batch shape times every candidate on `stream` (synchronously, so make that call
 * before any stream capture); later calls reuse the choice, which can be persisted in the
 * file named by SSE_AUTOTUNE_CACHE (SSE_AUTOTUNE=0 skips tuning).  After tuning, the call
 * is asynchronous and stream-ordered (it allocates its 4-byte work counter with
 * cudaMallocAsync on `stream`), so it can be captured in a CUDA graph.  Results equal those
 * of sse_execute on each instance alone, bit for bit.  Device-wait timeouts of every
 * instance are recorded in plans[0]'s status word (read it with sse_plan_status(plans[0])). */
SSE_API sse_status sse_execute_batch(sse_plan_t *const *plans, const sse_io *ios, int32_t n, void *stream);

/* The autotuner's choice for this batch shape: SSE_OK with the values, or SSE_NOT_READY
 * if the shape has not been tuned yet. */
SSE_API sse_status sse_batch_tuning(sse_plan_t *const *plans, const sse_io *ios, int32_t n, int32_t *tiles_per_unit,
                                    int32_t *longest_first);

/* ---- serving: a request loop with continuous batching ------------------------------------
 *
 * A server owns a host thread and two CUDA streams on the device current at creation, each
 * with its own device status word and work counter (allocated once, at creation).
 * Requests (a mixed-mode plan plus device buffers the caller keeps resident between SCBA
 * iterations) are admitted in arrival order while the admitted working set stays within
 * mem_budget_bytes and at most max_inflight requests are admitted.  The working set counts
 * each admitted request's resident bytes (G, Dt and Sigma of each requested sign) plus,
 * once per plan held by an admitted request, the device memory that plan owns (its status
 * word and tensor-core workspace).  Every admitted request that has not started joins the
 * next round: one persistent batched launch (as sse_execute_batch, with the tuned split
 * when the shape was tuned before, else the default split) on a stream that no running
 * round uses, so new arrivals start while older rounds drain.  A round's device-wait
 * timeouts are recorded in that round's own status word and reported on every ticket of
 * the round.  A ticket borrows its plan and buffers until sse_poll returns a final status. */
typedef struct {
    sse_status status;    /* final status once sse_poll stops returning SSE_NOT_READY */
    double t_submit_ms;   /* host steady-clock times (milliseconds) */
    double t_start_ms;    /* when its round's kernels had been enqueued (0 before) */
    double t_end_ms;      /* when the server saw its round complete (or cancelled it) */
    int32_t round_size;   /* requests in the round it ran in */
} sse_result;

/* wait_limit_ms bounds how long sse_server_shutdown / sse_server_destroy wait for running
 * rounds (0: 1000). */
SSE_API sse_status sse_server_create(uint64_t mem_budget_bytes, int32_t max_inflight, uint32_t wait_limit_ms,
                                     sse_server_t **out);
/* Non-blocking.  Precondition: every write to the request's input buffers (G, Dt) is
 * complete on the device before the call -- the server's streams do not wait for the
 * caller's streams (synchronise the stream that filled them, or wait on its event first).
 * SSE_E_OVER_BUDGET if the request and its plan's workspace alone exceed the budget (it
 * could never be admitted); SSE_E_SHUTDOWN after shutdown began. */
SSE_API sse_status sse_submit(sse_server_t *server, sse_plan_t *plan, const sse_io *io, uint64_t *ticket);
/* SSE_NOT_READY while queued or running; then the request's final status (SSE_OK, a CUDA
 * error, SSE_E_TIMEOUT if a device wait of its round expired, SSE_E_OUT_OF_MEMORY, or
 * SSE_E_CANCELLED), after which the ticket is forgotten and later polls give
 * SSE_E_UNKNOWN_TICKET.  `out` (may be NULL) receives status and timestamps. */
SSE_API sse_status sse_poll(sse_server_t *server, uint64_t ticket, sse_result *out);
/* Stops admitting, cancels every request that has not started (they end with
 * SSE_E_CANCELLED and stay pollable) and waits up to wait_limit_ms for running rounds:
 * SSE_OK once none runs, SSE_E_TIMEOUT otherwise.  Later submits give SSE_E_SHUTDOWN. */
SSE_API sse_status sse_server_shutdown(sse_server_t *server);
/* sse_server_shutdown, then frees the server (SSE_E_TIMEOUT, and the server is not freed,
 * if rounds are still running after wait_limit_ms). */
SSE_API sse_status sse_server_destroy(sse_server_t *server);
/* Rounds launched so far and the admitted working set (bytes, requests). */
SSE_API sse_status sse_server_stats(sse_server_t *server, uint64_t *rounds, uint64_t *inflight_bytes,
                                    int32_t *inflight);

/* Synchronise the plan's last stream and read (then clear) the device status word that
 * its kernels write: SSE_OK, SSE_E_TIMEOUT if a bounded device wait expired, or (only in
 * the bounds-checked build, libsse_gb300_bc.so) SSE_E_BOUNDS if a kernel computed an index
 * outside one of its buffers and skipped that access. */
SSE_API sse_status sse_plan_status(sse_plan_t *plan);

/* Kernel timing of sse_execute on one plan, for benchmarks and profiling; the paper has no
 * counterpart.  While enabled, every sse_execute call on the plan records three CUDA events
 * on its stream: before the workspace pass (the Nkz = 5 tensor-core form re-encodes G and
 * builds the slot tables there; other forms have none), before the main kernel and after
 * it.  enable != 0 starts timing and zeroes the totals (the first call creates the events);
 * 0 stops.  Batched and served executions are not timed. */
SSE_API sse_status sse_plan_set_timing(sse_plan_t *plan, int32_t enable);
/* Totals since timing was enabled: milliseconds spent in the workspace pass and in the
 * main kernel over `calls` timed calls.  Waits for the recorded events. */
SSE_API sse_status sse_plan_timing(sse_plan_t *plan, double *prep_ms, double *main_ms, int64_t *calls);

/* Mixed-mode evaluation for callers that cannot let this library allocate memory (for
 * example a framework whose allocator owns all device memory, or a loop that must not
 * stall on cudaMalloc/cudaFree).  No plan is created and nothing is allocated: the
 * neighbour list is range-checked on the device, and the little scratch the kernels
 * need (4 words: the check's result and the kernel's device-wait status) lives in one
 * fixed 256-byte device array built into the library, which every GPU that loads the
 * library keeps until the process exits.  The paper has no counterpart to this entry.
 * The first call on a device looks up that array's address; make it before any stream
 * capture.  All calls on a device share the array (each clears what it uses first), so
 * calls whose work overlaps on the GPU race.  Same arguments and results as sse_plan +
 * sse_execute in SSE_MODE_MIXED; geometries the mixed kernel cannot run (Nkz > 5,
 * nb_max > 32, or a shared-memory need beyond one SM) are rejected with
 * SSE_E_INVALID_ARG.  Every call synchronises `stream` twice (after the on-device
 * neighbour check, whose result it reads back, and at the end) and so blocks the calling
 * thread until Sigma is written; SSE_E_TIMEOUT if a bounded device wait expired. */
SSE_API sse_status sse_execute_noalloc(const sse_geometry *geo, const sse_io *io, void *stream);

/* Failure injection for tests of the failure detection; the paper has no counterpart.
 * Arms a one-shot, process-wide fault that the next matching event consumes:
 *   SSE_INJECT_STALL: the next launch of a mixed-mode kernel (sse_execute, sse_execute_batch
 *     or a server round) leaves one wait of each work unit's pipeline unsatisfied (the
 *     warp-specialised form skips the copy of a neighbour slot's operand tables; the other
 *     form skips the copy of one stage's G blocks).  The bounded device wait expires, the
 *     kernel drains what it has in flight, frees its tensor memory and returns; its status
 *     word reads SSE_E_TIMEOUT (sse_plan_status, sse_poll), Sigma is undefined, and the
 *     context stays usable.  Costs a few bounded waits of 0.25 s.
 *   SSE_INJECT_ALLOC_FAIL: the next per-request device allocation (a plan's workspace, the
 *     work counter of a batched launch) reports SSE_E_OUT_OF_MEMORY without allocating.
 *   SSE_INJECT_NONE: disarm. */
enum { SSE_INJECT_NONE = 0, SSE_INJECT_STALL = 1, SSE_INJECT_ALLOC_FAIL = 2 };
SSE_API sse_status sse_debug_inject(int32_t kind);

SSE_API const char *sse_status_string(sse_status status);
SSE_API const char *sse_last_error(void);
SSE_API int32_t sse_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SSE_GB300_SSE_H */
