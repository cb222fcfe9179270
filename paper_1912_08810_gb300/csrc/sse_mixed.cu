// Mixed-precision tensor-core forms of the electron scattering self-energy (Eq. 3).
//
// Regrouping used here (exact by linearity; Section 3 "Dataflow Optimizations" removes
// the (qz, w)-independent products from the correlation in the same spirit):
//   X_i[k', E']  = dH_i . G[k', E', f]                          (per slot b, f = neigh[a, b])
//   V_j[k, E]    = sum_{i, q, w} Dt_ij[q, w] X_i[(k-q) mod Nkz, E - w - omega_first]
//   Sigma[k, E] += sum_j V_j[k, E] . dH_j^dagger                (reduced over slots in FP64)
// The correlation is the dominant work.  It runs on the tensor cores (tcgen05, kind::f16)
// as a Toeplitz-in-E, circulant-in-k contraction (the matrix form of Section 3's nested
// map substitution): rows (k, j, e) of a tile of energies, K = (energy slot E' of the
// tile's window, i, k', re/im), N = the 144 channels (r, t) of a 12 x 12 block, two TMEM
// accumulators (Re V, Im V).  Operands are split into bf16 hi + lo and contracted as
// hi*hi + hi*lo + lo*hi with FP32 accumulation; each slot's FP32 result is added into
// Sigma in FP64 for complex128 output.
//
// Two kernels:
// - sse_tc_kernel (warp-specialised, every Nkz <= 5 when its tiles fit in shared memory):
//   the Toeplitz operand read in place from a per-(atom, slot) table by shifting the
//   descriptor, both small products (dH_i . G and V . dH_j^dagger) on the tensor cores too,
//   roles split over 16 warps (operand builders, three MMA-issuing lanes, a bulk-copy lane;
//   below Nkz = 5 the warps of TMEM lane quarter 3 encode raw G blocks for the pre-product);
//   fed by the workspace pass (sse_split_g_kernel at Nkz = 5, sse_slot_tables_kernel).
// - sse_mixed_kernel (single role, no workspace; sse_execute_noalloc, large Nw): one CTA
//   converts the stage's G blocks, builds X and the Toeplitz slice in shared memory with
//   FP32 CUDA-core products, issues the MMAs from one thread while the next stage is built,
//   and applies dH_j^dagger in FP32 on the CUDA cores at the end of each job.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdlib.h>

#include "sse_internal.h"
#include "tc_ptx.h"

namespace sse {
namespace {

using namespace tc;

constexpr int kThreads = 256;
constexpr int kRowsMax = 128;    // MMA M
constexpr int kCh = 144;         // MMA N: channels of a 12 x 12 block
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccIm = 256; // TMEM column of the imaginary accumulator
constexpr uint64_t kWaitNs = 250000000ull;  // bound on every device-side wait (0.25 s)
constexpr int kMaxSlots = 32;
constexpr int kVStride = 73;     // row stride (floats) of the drained accumulator tile

// Compile-time tile geometry for a given Nkz.
template <int NK>
struct Geo {
    static constexpr int KS = ((6 * NK + 7) / 8) * 8;  // K values per energy slot (i, k', re/im), padded
    static constexpr int P = (KS % 16 == 0) ? 1 : 2;   // energy slots per stage (stage K multiple of 16)
    static constexpr int KST = P * KS;                 // K per stage
    static constexpr int TE = kRowsMax / (3 * NK);     // energies per tile
    static constexpr int ROWS = 3 * NK * TE;           // used MMA rows
    static constexpr int SBO_B = (KST / 8) * 128;      // bytes between 8-row groups of B
    static constexpr int B_PLANE = (kCh / 8) * SBO_B;
    static constexpr int SBO_A = (KST / 8) * 128;
    static constexpr int A_PLANE = (kRowsMax / 8) * SBO_A;
    // Direct-descriptor form (Nkz = 5): rows (k, j, e) in groups of 8 energies, K per
    // energy slot = (i, k') padded to 16, Re/Im of X in separate B planes, and the
    // Toeplitz operand read in place from a per-slot table by shifting the descriptor.
    static constexpr bool DA = (NK == 5);
    static constexpr int DA_TE = 8;
    static constexpr int DA_K = 16;                    // (i, k') per slot, padded
    static constexpr int DA_SBO_B = (DA_K / 8) * 128;  // 256 bytes
    static constexpr int DA_B_PLANE = (kCh / 8) * DA_SBO_B;
    static constexpr int DA_GROUPS = 16;               // 8-row groups of the 128-row tile
};


// Re-encoded G for the tensor-core pre-product X = dH . G: one (E', f) slice holds rows
// (k', t) = 12 Nkz padded to 64 by K = (re/im of G, u) = 24 padded to 32, hi then lo plane.
constexpr int kXpSlice = 8192;

constexpr int kMaxInst = 64;  // instances per launch (the descriptors travel as kernel parameters)

// One independent SSE instance of a launch.  Its work is split into units
// (sign, atom, range of tiles); units are numbered from unit_begin.
struct InstDesc {
    const void *G[2];
    const void *D[2];
    void *S[2];
    const void *dH;
    const int32_t *neigh;
    int32_t na, ne, nb, nqz;
    int32_t ntiles;         // tiles per atom
    int32_t tiles_per_cta;  // tiles per unit
    int32_t nchunks;        // units per (sign, atom)
    int32_t nsign;
    long long unit_begin;
    const int32_t *rev;     // non-null: D holds the full phonon tensors and Dt is formed on the fly
    const uint8_t *gws[2];  // tensor-core form: G re-encoded per sign (see sse_split_g_kernel)
    const uint8_t *sws[2];  // tensor-core form: slot tables per sign (see sse_slot_tables_kernel)
};

struct MixParams {
    int32_t *status;        // device status word (bounded waits that expired)
    int32_t *queue;         // work counter of a persistent launch; null: unit = blockIdx.x
    int32_t nkz, nw, omega_first;
    int32_t nst;            // stages per job
    int32_t n_inst;
    int32_t inject;         // failure-injection test hook (sse_debug_inject): skip one copy per CTA
    long long total_units;
    uint32_t off_b, off_a, off_g, off_df, off_dh, off_bar, off_x, off_bp, g_stage;
    int32_t nbst;           // warp-specialised form: B buffers in flight (2 or 3)
    uint32_t off_stg;       // warp-specialised form, Nkz = 5: staged post-product results (0: none)
    InstDesc inst[kMaxInst];
};

template <typename CT>
__device__ __forceinline__ double2 ld_c64(const CT *p);
template <>
__device__ __forceinline__ double2 ld_c64<double2>(const double2 *p) { return __ldg(p); }
template <>
__device__ __forceinline__ double2 ld_c64<float2>(const float2 *p) {
    const float2 v = __ldg(p);
    return make_double2(f32_to_f64(v.x), f32_to_f64(v.y));
}

// Entry ij of Dt[q, w, a, b] in FP32.  Without `rev`, D holds Dt [nqz][nw][na][nb][3][3];
// with it, D holds the full phonon tensor [nqz][nw][na][nb + 1][3][3] (block nb = D_aa) and
// the pre-combination of Eq. 3, Dt = ((D_ba - D_bb) - D_aa) + D_ab with D_ba the block of
// f = neigh[a, b] at its slot rev[a, b], is formed here in FP64 and rounded once -- the
// same value the stand-alone pre-combination kernel stores.  Only for slots with f >= 0.
template <typename CT>
__device__ __forceinline__ float2 load_dt(const CT *__restrict__ D, const int32_t *__restrict__ neigh,
                                          const int32_t *__restrict__ rev, int q, int w, int nw, int na, int nb,
                                          int a, int b, int ij, int32_t *status) {
    if (!rev) return load_c32(D + ((((size_t)q * nw + w) * na + a) * nb + b) * 9 + ij);
    const size_t qw = ((size_t)q * nw + w) * na;
    const int f = __ldg(neigh + (size_t)a * nb + b), r = __ldg(rev + (size_t)a * nb + b);
    if (!SSE_BC(f, na, status) || !SSE_BC(r, nb, status)) return make_float2(0.f, 0.f);
    const size_t nb1 = (size_t)nb + 1;
    const double2 ab = ld_c64(D + ((qw + a) * nb1 + b) * 9 + ij), aa = ld_c64(D + ((qw + a) * nb1 + nb) * 9 + ij);
    const double2 ba = ld_c64(D + ((qw + f) * nb1 + r) * 9 + ij), bb = ld_c64(D + ((qw + f) * nb1 + nb) * 9 + ij);
    const double x = ((ba.x - bb.x) - aa.x) + ab.x, y = ((ba.y - bb.y) - aa.y) + ab.y;
    return make_float2(f64_to_f32(x), f64_to_f32(y));
}

__device__ __forceinline__ float2 cmul_conj_acc(float2 acc, float2 v, float2 h) {
    // acc + v * conj(h)
    acc.x = fmaf(v.x, h.x, acc.x);
    acc.x = fmaf(v.y, h.y, acc.x);
    acc.y = fmaf(v.y, h.x, acc.y);
    acc.y = fmaf(-v.x, h.y, acc.y);
    return acc;
}

// (hi, lo) bf16 splits of two floats, packed: .x = (hi(a), hi(b)), .y = (lo(a), lo(b)),
// the first value in the low half of each word.
__device__ __forceinline__ uint2 split2_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    return make_uint2(*reinterpret_cast<const uint32_t *>(&h), *reinterpret_cast<const uint32_t *>(&l));
}

// Split products folded into K (Nkz <= 3, where a K row (i, k') holds L = 3 Nkz <= 9 values):
// the row x becomes [hi(x) | hi(x) | lo(x) | 0] on one side of the MMA and [hi | lo | hi | 0]
// on the other, so that one K = 32 contraction gives hi.hi + hi.lo + lo.hi.  `first_hi`
// selects the [hi | hi | lo] order (the Toeplitz operand); otherwise [hi | lo | hi] (X).
// Returns the 32 bf16 values packed in pairs, the first in the low half of each word.
template <int L>
__device__ __forceinline__ void splitk_row(const float *x, bool first_hi, uint32_t (&w)[16]) {
    static_assert(3 * L <= 32, "split-in-K row");
    uint32_t h[L], l[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const __nv_bfloat16 hb = __float2bfloat16_rn(x[i]);
        const __nv_bfloat16 lb = __float2bfloat16_rn(x[i] - __bfloat162float(hb));
        h[i] = __bfloat16_as_ushort(hb);
        l[i] = __bfloat16_as_ushort(lb);
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        uint32_t pair = 0;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int kk = 2 * m + half, seg = kk / L, idx = kk % L;
            uint32_t v = 0;
            if (seg == 0) v = h[idx];
            else if (seg == 1) v = first_hi ? h[idx] : l[idx];
            else if (seg == 2) v = first_hi ? l[idx] : h[idx];
            pair |= v << (16 * half);
        }
        w[m] = pair;
    }
}

// Each word holds a (re-part, im-part) K pair (Re T, -Im T); the imaginary-part accumulator
// needs (Im T, Re T): swap the halves and flip the sign of the new low half.
__device__ __forceinline__ uint32_t to_im_pair(uint32_t w) { return __byte_perm(w, 0u, 0x1032) ^ 0x00008000u; }
__device__ __forceinline__ uint4 to_im_pairs(uint4 v) {
    return make_uint4(to_im_pair(v.x), to_im_pair(v.y), to_im_pair(v.z), to_im_pair(v.w));
}

// G of one sign re-encoded for the tensor-core pre-product: slice (E', f) holds, for rows
// n' = (t / 4) * 4 Nkz + k' * 4 + t % 4 (12 Nkz used, 64 rows) and K = pc * 12 + u (24 used,
// 32), the bf16 hi plane then the lo plane of the pc-part of G[k', E', f][u, t], in the
// K-major core-matrix layout (SBO 512, LBO 128).  One CTA per slice.  The row order makes a
// 16-lane TMEM load of the product hand each builder thread whole K rows of the main MMA's B.
template <typename CT>
__global__ void __launch_bounds__(256) sse_split_g_kernel(const CT *__restrict__ G, uint8_t *__restrict__ ws,
                                                          int ne, int na, int nkz) {
    __shared__ float2 sg[5 * kCh];  // G[k', E', f] of the slice (Nkz = 5), read contiguously
    if (nkz > 5) return;           // stored slices serve Nkz = 5 only (below, the kernel encodes G)
    const long long slice = blockIdx.x;
    const int E = (int)(slice / na), f = (int)(slice % na);
    for (int x = threadIdx.x; x < nkz * kCh; x += 256)
        sg[x] = load_c32(G + (((size_t)(x / kCh) * ne + E) * na + f) * kCh + x % kCh);
    __syncthreads();
    const int np = threadIdx.x >> 2, kg = threadIdx.x & 3;
    float v[8];
#pragma unroll
    for (int xx = 0; xx < 8; ++xx) {
        const int kk = kg * 8 + xx;
        float val = 0.f;
        if (np < nkz * 12 && kk < 24) {
            const int blk = np / (4 * nkz), kp = (np % (4 * nkz)) / 4, t = 4 * blk + np % 4;
            const int pc = kk / 12, u = kk % 12;
            const float2 c = sg[kp * kCh + u * 12 + t];
            val = pc ? c.y : c.x;
        }
        v[xx] = val;
    }
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int xx = 0; xx < 4; ++xx) {
        const uint2 hl = split2_bf16(v[2 * xx], v[2 * xx + 1]);
        hv[xx] = hl.x;
        lv[xx] = hl.y;
    }
    uint8_t *dst = ws + slice * 8192 + (np >> 3) * 512 + kg * 128 + (np & 7) * 16;
    *(uint4 *)dst = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    *(uint4 *)(dst + 4096) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

// Sigma after one more slot: the slot's FP32 contribution v added in FP64 to the value
// stored so far (old), or v alone for the first slot.
template <typename CT>
__device__ __forceinline__ CT slot_sum(float2 v, CT old, bool first);
template <>
__device__ __forceinline__ double2 slot_sum<double2>(float2 v, double2 old, bool first) {
    double2 o = make_double2(f32_to_f64(v.x), f32_to_f64(v.y));
    if (!first) {
        o.x += old.x;
        o.y += old.y;
    }
    return o;
}
template <>
__device__ __forceinline__ float2 slot_sum<float2>(float2 v, float2 old, bool first) {
    if (first) return v;
    const double x = f32_to_f64(old.x) + f32_to_f64(v.x);
    const double y = f32_to_f64(old.y) + f32_to_f64(v.y);
    return make_float2(f64_to_f32(x), f64_to_f32(y));
}

// Sum over neighbour slots in the warp-specialised form: the first slot's contribution is
// stored in the output type; each later slot's FP32 contribution is added in place by a
// reduction at L2 -- widened exactly and added in FP64 for complex128 output (the running
// sum over slots is an FP64 sum), added in FP32 for complex64 output (the output's own
// precision).
template <typename CT>
__device__ __forceinline__ CT final_of(float2 v);
template <>
__device__ __forceinline__ double2 final_of<double2>(float2 v) { return make_double2(f32_to_f64(v.x), f32_to_f64(v.y)); }
template <>
__device__ __forceinline__ float2 final_of<float2>(float2 v) { return v; }
__device__ __forceinline__ void slot_add(double2 *p, float2 v) { red_add_f64x2(p, f32_to_f64(v.x), f32_to_f64(v.y)); }
__device__ __forceinline__ void slot_add(float2 *p, float2 v) { red_add_f2(p, v); }

template <int NK, typename CT>
__global__ void __launch_bounds__(kThreads, 1) sse_mixed_kernel(const __grid_constant__ MixParams prm) {
    using GG = Geo<NK>;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nw = prm.nw;
    const int omega_max = prm.omega_first + nw - 1;
    const int nw0 = nw + GG::P - 1;                   // rows of the table per (k, j)
    const int da_rows = nw + 2 * GG::DA_TE - 2;       // direct table: rows w0 + (TE - 1), w0 in [1-TE, nw+TE-2]
    constexpr uint32_t tab_stride = GG::KST * 4 + 16;  // hi + lo + 16 bytes against bank conflicts
    // (k, j) groups of rows: padded so that consecutive groups -- read by consecutive lanes --
    // start 16 bytes apart modulo 128 and the 16-byte loads of 8 lanes hit distinct banks
    const uint32_t grp_stride = ((uint32_t)nw0 * tab_stride + 127u) / 128u * 128u + 16u;

    uint8_t *sB = smem + prm.off_b;                 // [2 stages][hi, lo] B planes
    uint8_t *sA = smem + prm.off_a;                 // [2 stages][re, im][hi, lo] A planes
    uint8_t *sG = smem + prm.off_g;                 // [2 stages] raw G blocks
    uint8_t *sTab = smem + prm.off_df;                // Toeplitz row table of the current slot
    float2 *sDh = (float2 *)(smem + prm.off_dh);      // [3][144] fp32 dH of the current slot
    // Jobs (tile, slot) of a unit run slot-major, so the per-slot tables are built once per
    // slot and reused by the unit's tiles; the direct form keeps tile-major order because its
    // drained accumulators overlay the direct table.
    constexpr bool SLOT_OUTER = !GG::DA;
    // epilogue: the accumulators are drained in EP_PARTS column blocks of EP_R rows r
    constexpr int EP_PARTS = 2;
    constexpr int EP_COLS = kCh / EP_PARTS, EP_STRIDE = EP_COLS + 1, EP_R = EP_COLS / 12;
    constexpr int EP_RB = EP_R / 2, EP_NSB = 6 / EP_RB, EP_S = 12 / EP_NSB;
    static_assert(EP_STRIDE * 2 * kRowsMax * 4 <= 2 * kRowsMax * kVStride * 4, "drain buffer");
    // drained accumulators: overlay B and A, or (direct form) the per-slot table
    float *sV = (float *)(GG::DA ? smem + prm.off_df : smem + prm.off_b);
    static_assert(!GG::DA || GG::TE == GG::DA_TE, "direct form expects 8 energies per tile");
    uint64_t *bar_mma = (uint64_t *)(smem + prm.off_bar);
    uint64_t *bar_g = bar_mma + 2;                   // [3] (two used without the pre-product)
    uint64_t *bar_job = bar_mma + 5;
    uint64_t *bar_fin = bar_mma + 6;                 // only for draining MMAs on abort
    uint32_t *s_tmem = (uint32_t *)(bar_mma + 9);
    int *s_abort = (int *)(s_tmem + 1);
    int *s_nvalid = s_abort + 1;
    long long *s_unit = (long long *)(smem + prm.off_bar + 128);
    int *s_slot = (int *)(s_unit + 1);                // [kMaxSlots] valid slot indices
    int *s_f = s_slot + kMaxSlots;                    // [kMaxSlots] their neighbour atoms

    if (tid == 0) {
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        mbar_init(&bar_g[0], 1);
        mbar_init(&bar_g[1], 1);
        mbar_init(&bar_g[2], 1);
        mbar_init(bar_job, 1);
        mbar_init(bar_fin, 1);
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == 0) {
        tmem_alloc(s_tmem, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    // Per-thread A-builder row: thread -> (accumulator q, row m).
    const int aq = tid >> 7, am = tid & 127;
    const bool arow_ok = am < GG::ROWS;
    const int ae = am / (3 * NK), ak = (am / 3) % NK, aj = am % 3;

    bool abort = false;
    int abort_g = -1, abort_total = 0;
    int g_base = 0;   // stages this CTA ran before the current unit
    int job_ctr = 0;  // jobs this CTA completed (phase of the job barrier)
    for (long long iter = 0;; ++iter) {
    // ---- next unit: one per CTA, or pulled from the work counter ----
    __syncthreads();
    if (tid == 0) {
        long long u;
        if (prm.queue) u = atomicAdd(prm.queue, 1);
        else u = iter == 0 ? (long long)blockIdx.x : prm.total_units;
        if (*(volatile int32_t *)prm.status != 0) u = prm.total_units;  // another CTA timed out
        *s_unit = u;
    }
    __syncthreads();
    const long long unit = *s_unit;
    if (unit >= prm.total_units) break;
    int ii = 0;
    while (ii + 1 < prm.n_inst && prm.inst[ii + 1].unit_begin <= unit) ++ii;
    const InstDesc &I = prm.inst[ii];
    const long long local = unit - I.unit_begin;
    const int sign = (int)(local / ((long long)I.na * I.nchunks));
    const long long rem = local - (long long)sign * I.na * I.nchunks;
    const int a = (int)(rem / I.nchunks), chunk = (int)(rem % I.nchunks);
    const Dims d{prm.nkz, I.nqz, I.ne, nw, I.na, I.nb, prm.omega_first};
    const CT *__restrict__ G = (const CT *)I.G[sign];
    const CT *__restrict__ D = (const CT *)I.D[sign];
    CT *__restrict__ S = (CT *)I.S[sign];
    const CT *__restrict__ dH = (const CT *)I.dH;
    const int t_begin = chunk * I.tiles_per_cta;
    const int t_end = min(I.ntiles, t_begin + I.tiles_per_cta);

    if (tid == 0) {
        int nv = 0;
        for (int b = 0; b < d.nb && nv < kMaxSlots; ++b) {
            const int f = __ldg(I.neigh + (size_t)a * d.nb + b);
            if (f >= 0) {
                s_slot[nv] = b;
                s_f[nv] = f;
                ++nv;
            }
        }
        *s_nvalid = nv;
    }
    __syncthreads();
    const int nvalid = *s_nvalid;
    const int njobs = (t_end - t_begin) * nvalid;
    const int total = njobs * prm.nst;

    if (nvalid == 0) {
        // no neighbours: Sigma is zero on this unit's points
        for (int t = t_begin; t < t_end; ++t)
            for (int x = tid; x < NK * GG::TE * kCh; x += kThreads) {
                const int e = x / (NK * kCh), k = (x / kCh) % NK, c = x % kCh;
                const int E = t * GG::TE + e;
                if (E < d.ne) {
                    CT z;
                    z.x = 0;
                    z.y = 0;
                    S[(((size_t)k * d.ne + E) * d.na + a) * kCh + c] = z;
                }
            }
    }

    // Position of a stage in the unit: (tile, valid-slot index, stage within the job),
    // stepped forward without divisions.
    struct Pos {
        int t, vs, st;
    };
    auto advance = [&](Pos &p) {
        if (++p.st < prm.nst) return;
        p.st = 0;
        if constexpr (SLOT_OUTER) {
            if (++p.t == t_end) {
                p.t = t_begin;
                ++p.vs;
            }
        } else {
            if (++p.vs == nvalid) {
                p.vs = 0;
                ++p.t;
            }
        }
    };
    // Thread 0: bulk-copy the G blocks of stage g (at position q) into raw buffer g % 2.
    // The failure-injection hook leaves the second stage of the CTA's first unit uncopied.
    auto issue_g = [&](int g, const Pos &q) {
        if (prm.inject && iter == 0 && g == (total > 1 ? 1 : 0)) return;
        const int t = q.t, vs = q.vs, st = q.st;
        const int f = s_f[vs];
        const int e_first = t * GG::TE - omega_max + GG::P * st;
        uint32_t bytes = 0;
#pragma unroll
        for (int p = 0; p < GG::P; ++p) {
            const int Ep = e_first + p;
            if (Ep >= 0 && Ep < d.ne) bytes += NK * kCh * (uint32_t)sizeof(CT);
        }
        const int gg = g_base + g;
        uint64_t *bar = &bar_g[gg & 1];
        mbar_arrive_expect_tx(bar, bytes);
        uint8_t *dst = sG + (gg & 1) * prm.g_stage;
#pragma unroll
        for (int p = 0; p < GG::P; ++p) {
            const int Ep = e_first + p;
            if (Ep < 0 || Ep >= d.ne) continue;
            for (int kp = 0; kp < NK; ++kp) {
                const size_t src = (((size_t)kp * d.ne + Ep) * d.na + f) * kCh;
                // a skipped copy leaves the stage's barrier short: its wait then times out
                if (SSE_BC(src + kCh - 1, (long long)d.nkz * d.ne * d.na * kCh, prm.status))
                    bulk_g2s(dst + (p * NK + kp) * kCh * sizeof(CT), G + src, kCh * (uint32_t)sizeof(CT), bar);
            }
        }
    };

    Pos cur{t_begin, 0, 0};  // the stage being built
    Pos pf{t_begin, 0, 0};   // thread 0: the next stage to prefetch
    if (tid == 0 && total > 0) issue_g(0, pf), advance(pf);

    for (int g = 0; g < total && !abort; ++g, advance(cur)) {
        const int t = cur.t, vs = cur.vs, st = cur.st;
        const int gg = g_base + g;  // CTA-wide stage index: buffer and barrier phases
        const int sb = gg & 1;
        const int E0 = t * GG::TE;
        const bool job_first = st == 0, job_last = st == prm.nst - 1;
        // first stage of a slot's first job
        const bool slot_first = job_first && (!SLOT_OUTER || t == t_begin);

        // another CTA timed out: stop early instead of waiting out every bound
        if (job_first && tid == 0 && *(volatile int32_t *)prm.status != 0) *s_abort = 1;
        if (slot_first) {
            // Slot tables: dH (fp32) and the folded, split, k-rotated Dt.  The previous
            // job's MMAs are complete, so the B (and A) stages are free scratch.
            const int b = s_slot[vs];
            const CT *dh = dH + ((size_t)a * d.nb + b) * 3 * kCh;
            for (int x = tid; x < 3 * kCh; x += kThreads)
                sDh[x] = SSE_BC((dh - dH) + x, (long long)d.na * d.nb * 3 * kCh, prm.status) ? load_c32(dh + x)
                                                                                           : make_float2(0.f, 0.f);
            float2 *dfold = (float2 *)sB;  // [kappa][w][ij] folded Dt (fp32), A/B area as scratch
            for (int x = tid; x < NK * nw * 9; x += kThreads) {
                const int ij = x % 9, w = (x / 9) % nw, kap = x / (9 * nw);
                // fold qz onto kz' = qz mod Nkz: T depends on (k - k') mod Nkz only
                float2 acc = make_float2(0.f, 0.f);
                for (int q = kap; q < d.nqz; q += NK) {
                    const float2 v = load_dt(D, I.neigh, I.rev, q, w, nw, d.na, d.nb, a, b, ij, prm.status);
                    acc.x += v.x;
                    acc.y += v.y;
                }
                dfold[x] = acc;
            }
            __syncthreads();
            if constexpr (GG::DA) {
                // Direct table: [q = Re, Im][hi, lo][group g = (k, j)][K group][row r] x 16 bytes,
                // entry (i, k') of row r = Re or Im of Df_ij[(k - k') mod Nkz][r - (TE - 1)].
                const int nitems = 2 * 2 * GG::DA_GROUPS * 2 * da_rows / 2;  // (q, g, kg, r): hi and lo together
                for (int x = tid; x < nitems; x += kThreads) {
                    const int r = x % da_rows, kg = (x / da_rows) % 2, g = (x / (2 * da_rows)) % GG::DA_GROUPS;
                    const int q = x / (2 * da_rows * GG::DA_GROUPS);
                    const int k = g / 3, j = g % 3, w0 = r - (GG::DA_TE - 1);
                    float v[8];
#pragma unroll
                    for (int xx = 0; xx < 8; ++xx) {
                        const int kk = kg * 8 + xx;
                        float val = 0.f;
                        if (g < 3 * NK && kk < 3 * NK && w0 >= 0 && w0 < nw) {
                            const int i = kk / NK, kp = kk % NK;
                            const float2 T = dfold[(((k - kp + NK) % NK) * nw + w0) * 9 + i * 3 + j];
                            val = q ? T.y : T.x;
                        }
                        v[xx] = val;
                    }
                    uint32_t hv[4], lv[4];
#pragma unroll
                    for (int xx = 0; xx < 4; ++xx) {
                        const uint2 hl = split2_bf16(v[2 * xx], v[2 * xx + 1]);
                        hv[xx] = hl.x;
                        lv[xx] = hl.y;
                    }
                    const size_t base_hi = ((((size_t)(q * 2 + 0) * GG::DA_GROUPS + g) * 2 + kg) * da_rows + r) * 16;
                    const size_t base_lo = ((((size_t)(q * 2 + 1) * GG::DA_GROUPS + g) * 2 + kg) * da_rows + r) * 16;
                    *(uint4 *)(sTab + base_hi) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                    *(uint4 *)(sTab + base_lo) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                }
                __syncthreads();
            } else {
            // Row table of the real-part accumulator's Toeplitz operand: one row per
            // (k, j, w0), w0 in [0, nw0); entry (p, i, k', re/im) = (Re T, -Im T) with
            // T = Df_ij[(k - k') mod Nkz][w0 - p]; bf16 hi plane then lo plane.  A tile row
            // (e, k, j) of stage st is the row w0 = e + nw - 1 - P * st.
            for (int x = tid; x < 3 * NK * nw0 * (GG::KST / 8); x += kThreads) {
                const int gq = x % (GG::KST / 8), row = x / (GG::KST / 8);
                const int w0 = row % nw0, kj = row / nw0, k = kj / 3, j = kj % 3;
                uint32_t hv[4], lv[4];
#pragma unroll
                for (int xx = 0; xx < 8; xx += 2) {
                    float v2[2];
#pragma unroll
                    for (int y = 0; y < 2; ++y) {
                        const int kk = gq * 8 + xx + y;
                        const int pp = kk / GG::KS, r2 = kk % GG::KS;
                        float v = 0.f;
                        if (r2 < 6 * NK) {
                            const int pair = r2 >> 1, pc = r2 & 1, i = pair / NK, kp = pair % NK;
                            const int w = w0 - pp;
                            if (w >= 0 && w < nw) {
                                const float2 T = dfold[(((k - kp + NK) % NK) * nw + w) * 9 + i * 3 + j];
                                v = pc ? -T.y : T.x;
                            }
                        }
                        v2[y] = v;
                    }
                    const uint2 hl = split2_bf16(v2[0], v2[1]);
                    hv[xx / 2] = hl.x;
                    lv[xx / 2] = hl.y;
                }
                uint8_t *trow = sTab + (size_t)kj * grp_stride + (size_t)w0 * tab_stride;
                *(uint4 *)(trow + gq * 16) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                *(uint4 *)(trow + GG::KST * 2 + gq * 16) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
            }
            __syncthreads();
            }
        }

        uint8_t *gbuf = sG + sb * prm.g_stage;
        float2 *g32 = (float2 *)gbuf;  // [p][k'][u][t] complex fp32
        if (tid == 0 && g + 1 < total) issue_g(g + 1, pf), advance(pf);

        // ---- G blocks of this stage: wait, convert to fp32 in place, zero the gaps ----
        if (!mbar_wait_bounded(&bar_g[sb], (gg >> 1) & 1, kWaitNs)) {
            *s_abort = 1;
            atomicOr(prm.status, kStatusTimeout);
        }
        {
            constexpr int NE_ = GG::P * NK * kCh;
            constexpr int PER = (NE_ + kThreads - 1) / kThreads;
            float2 v[PER];
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int x = tid + r * kThreads;
                v[r] = make_float2(0.f, 0.f);
                if (x < NE_) {
                    const int p = x / (NK * kCh);
                    const int Ep = E0 - omega_max + GG::P * st + p;
                    if (Ep >= 0 && Ep < d.ne) {
                        if (sizeof(CT) == 16) {
                            const double2 raw = ((const double2 *)gbuf)[x];
                            v[r] = make_float2(f64_to_f32(raw.x), f64_to_f32(raw.y));
                        } else {
                            v[r] = ((const float2 *)gbuf)[x];
                        }
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int x = tid + r * kThreads;
                if (x < NE_) g32[x] = v[r];
            }
        }

        // ---- the stage buffers must be free: MMAs of stage g - 2 complete ----
        if (gg >= 2 && !mbar_wait_bounded(&bar_mma[sb], ((gg >> 1) - 1) & 1, kWaitNs)) {
            *s_abort = 1;
            atomicOr(prm.status, kStatusTimeout);
        }
        __syncthreads();

        uint8_t *bhi = sB + sb * (2 * GG::B_PLANE), *blo = bhi + GG::B_PLANE;
        uint8_t *abase = sA + sb * (4 * GG::A_PLANE);
        uint8_t *bda = sB + sb * (4 * GG::DA_B_PLANE);  // direct form: [re, im][hi, lo] planes

        // ---- X slices: X_i[k'][r, t] = sum_u dH_i[r, u] G[k'][u, t] -> B (bf16 hi / lo) ----
        for (int item = tid; item < GG::P * kCh; item += kThreads) {
            const int p = item / kCh, n = item % kCh, r = n / 12, tt = n % 12;
            uint32_t hw[GG::KS / 2], lw[GG::KS / 2];
#pragma unroll
            for (int x = 0; x < GG::KS / 2; ++x) {
                hw[x] = 0u;
                lw[x] = 0u;
            }
            float2 hrow[3][12];  // dH_i[r, :] for the three directions
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int u = 0; u < 12; ++u) hrow[i][u] = sDh[i * kCh + r * 12 + u];
#pragma unroll
            for (int kp = 0; kp < NK; ++kp) {
                const float2 *gcol = g32 + (p * NK + kp) * kCh + tt;
                float xr[3] = {0.f, 0.f, 0.f}, xi[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int u = 0; u < 12; ++u) {
                    const float2 gv = gcol[u * 12];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        xr[i] = fmaf(hrow[i][u].x, gv.x, xr[i]);
                        xr[i] = fmaf(-hrow[i][u].y, gv.y, xr[i]);
                        xi[i] = fmaf(hrow[i][u].x, gv.y, xi[i]);
                        xi[i] = fmaf(hrow[i][u].y, gv.x, xi[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const uint2 hl = split2_bf16(xr[i], xi[i]);  // K index 2 * pair (re), 2 * pair + 1 (im)
                    hw[i * NK + kp] = hl.x;
                    lw[i * NK + kp] = hl.y;
                }
            }
            if constexpr (GG::DA) {
                // de-interleave: K index i * Nkz + k' of the Re and Im planes
                uint32_t hre[8], lre[8], him[8], lim[8];
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const uint32_t h0 = 2 * x < 3 * NK ? hw[2 * x] : 0u, h1 = 2 * x + 1 < 3 * NK ? hw[2 * x + 1] : 0u;
                    const uint32_t l0 = 2 * x < 3 * NK ? lw[2 * x] : 0u, l1 = 2 * x + 1 < 3 * NK ? lw[2 * x + 1] : 0u;
                    hre[x] = __byte_perm(h0, h1, 0x5410);
                    him[x] = __byte_perm(h0, h1, 0x7632);
                    lre[x] = __byte_perm(l0, l1, 0x5410);
                    lim[x] = __byte_perm(l0, l1, 0x7632);
                }
                const uint32_t row_off = (n >> 3) * GG::DA_SBO_B + (n & 7) * 16;
#pragma unroll
                for (int gq = 0; gq < 2; ++gq) {
                    const uint32_t o = row_off + gq * 128;
                    *(uint4 *)(bda + 0 * GG::DA_B_PLANE + o) = make_uint4(hre[4 * gq], hre[4 * gq + 1], hre[4 * gq + 2], hre[4 * gq + 3]);
                    *(uint4 *)(bda + 1 * GG::DA_B_PLANE + o) = make_uint4(lre[4 * gq], lre[4 * gq + 1], lre[4 * gq + 2], lre[4 * gq + 3]);
                    *(uint4 *)(bda + 2 * GG::DA_B_PLANE + o) = make_uint4(him[4 * gq], him[4 * gq + 1], him[4 * gq + 2], him[4 * gq + 3]);
                    *(uint4 *)(bda + 3 * GG::DA_B_PLANE + o) = make_uint4(lim[4 * gq], lim[4 * gq + 1], lim[4 * gq + 2], lim[4 * gq + 3]);
                }
            } else {
                const uint32_t row_off = (n >> 3) * GG::SBO_B + (n & 7) * 16 + (p * GG::KS / 8) * 128;
#pragma unroll
                for (int gq = 0; gq < GG::KS / 8; ++gq) {
                    *(uint4 *)(bhi + row_off + gq * 128) = make_uint4(hw[4 * gq], hw[4 * gq + 1], hw[4 * gq + 2], hw[4 * gq + 3]);
                    *(uint4 *)(blo + row_off + gq * 128) = make_uint4(lw[4 * gq], lw[4 * gq + 1], lw[4 * gq + 2], lw[4 * gq + 3]);
                }
            }
        }

        // ---- Toeplitz slice: A_q[(e, k, j), (p, i, k', re/im)] copied from the row table ----
        if constexpr (!GG::DA) {
            uint8_t *ahi = abase + aq * (2 * GG::A_PLANE), *alo = ahi + GG::A_PLANE;
            const uint32_t row_off = (am >> 3) * GG::SBO_A + (am & 7) * 16;
            const int w0 = ae + nw - 1 - GG::P * st;
            const bool live = arow_ok && w0 >= 0 && w0 < nw0;
            const uint8_t *trow = sTab + (size_t)(ak * 3 + aj) * grp_stride + (size_t)(live ? w0 : 0) * tab_stride;
#pragma unroll
            for (int gq = 0; gq < GG::KST / 8; ++gq) {
                uint4 h = make_uint4(0u, 0u, 0u, 0u), l = h;
                if (live) {
                    h = *(const uint4 *)(trow + gq * 16);
                    l = *(const uint4 *)(trow + GG::KST * 2 + gq * 16);
                    if (aq) {  // imaginary-part accumulator: (Im T, Re T) from (Re T, -Im T)
                        h = to_im_pairs(h);
                        l = to_im_pairs(l);
                    }
                }
                *(uint4 *)(ahi + row_off + gq * 128) = h;
                *(uint4 *)(alo + row_off + gq * 128) = l;
            }
        }

        fence_proxy_async_smem();
        __syncthreads();
        if (*s_abort) {
            abort = true;
            abort_g = gg;
            abort_total = g_base + total;
            break;
        }

        // ---- MMAs of this stage (one thread) ----
        if (tid == 0) {
            tc_fence_after();
            if constexpr (GG::DA) {
                // A: windows of the direct table starting at row (nw - 1 - st) + (TE - 1)
                constexpr uint32_t idesc = idesc_bf16_f32(kRowsMax, kCh);
                constexpr uint32_t idesc_negb = idesc | (1u << 14);
                const uint32_t lbo_a = (uint32_t)da_rows * 16, sbo_a = 2u * lbo_a;
                const uint32_t r_start = (uint32_t)(nw - 1 - st + GG::DA_TE - 1);
                const uint32_t tab0 = smem_u32(sTab) + r_start * 16;
                const uint32_t tstride = (uint32_t)GG::DA_GROUPS * 2 * da_rows * 16;  // one (q, split) table
                auto adesc = [&](int q, int split) {
                    return smem_desc(tab0 + (uint32_t)(q * 2 + split) * tstride, lbo_a, sbo_a);
                };
                const uint32_t b0 = smem_u32(bda);
                auto bdesc = [&](int q, int split) {
                    return smem_desc(b0 + (uint32_t)(q * 2 + split) * GG::DA_B_PLANE, 128, GG::DA_SBO_B);
                };
                const uint64_t are_h = adesc(0, 0), are_l = adesc(0, 1), aim_h = adesc(1, 0), aim_l = adesc(1, 1);
                const uint64_t bre_h = bdesc(0, 0), bre_l = bdesc(0, 1), bim_h = bdesc(1, 0), bim_l = bdesc(1, 1);
                const uint32_t dre = tmem, dim = tmem + kAccIm;
                // Re V = Re T Re X - Im T Im X
                mma_ss(dre, are_h, bre_h, idesc, job_first ? 0u : 1u);
                mma_ss(dre, are_h, bre_l, idesc, 1u);
                mma_ss(dre, are_l, bre_h, idesc, 1u);
                mma_ss(dre, aim_h, bim_h, idesc_negb, 1u);
                mma_ss(dre, aim_h, bim_l, idesc_negb, 1u);
                mma_ss(dre, aim_l, bim_h, idesc_negb, 1u);
                // Im V = Im T Re X + Re T Im X
                mma_ss(dim, aim_h, bre_h, idesc, job_first ? 0u : 1u);
                mma_ss(dim, aim_h, bre_l, idesc, 1u);
                mma_ss(dim, aim_l, bre_h, idesc, 1u);
                mma_ss(dim, are_h, bim_h, idesc, 1u);
                mma_ss(dim, are_h, bim_l, idesc, 1u);
                mma_ss(dim, are_l, bim_h, idesc, 1u);
            } else {
                constexpr uint32_t idesc = idesc_bf16_f32(kRowsMax, kCh);
                const uint32_t bh0 = smem_u32(bhi), bl0 = smem_u32(blo);
#pragma unroll
                for (int ks = 0; ks < GG::KST / 16; ++ks) {
                    const uint64_t bdh = smem_desc(bh0 + ks * 256, 128, GG::SBO_B);
                    const uint64_t bdl = smem_desc(bl0 + ks * 256, 128, GG::SBO_B);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const uint32_t ah = smem_u32(abase + q * (2 * GG::A_PLANE)) + ks * 256;
                        const uint64_t adh = smem_desc(ah, 128, GG::SBO_A);
                        const uint64_t adl = smem_desc(ah + GG::A_PLANE, 128, GG::SBO_A);
                        const uint32_t dt = tmem + (q ? kAccIm : 0u);
                        mma_ss(dt, adh, bdh, idesc, (job_first && ks == 0) ? 0u : 1u);
                        mma_ss(dt, adh, bdl, idesc, 1u);
                        mma_ss(dt, adl, bdh, idesc, 1u);
                    }
                }
            }
            mma_commit(&bar_mma[sb]);
            if (job_last) mma_commit(bar_job);
        }

        if (!job_last) continue;

        // ---- epilogue of the job: V = acc_re + i acc_im, Sigma += sum_j V_j dH_j^+ ----
        if (!mbar_wait_bounded(bar_job, job_ctr & 1, kWaitNs)) {
            *s_abort = 1;
            atomicOr(prm.status, kStatusTimeout);
        }
        tc_fence_after();
        ++job_ctr;
        const bool first_slot = vs == 0;
        for (int h = 0; h < EP_PARTS; ++h) {
            // the slots summed so far, fetched before the drain so their latency overlaps it
            const int ep_pt = tid / 6, ep_rb = (tid % 6) / EP_NSB, ep_sbk = (tid % 6) % EP_NSB;
            const int ep_e = ep_pt / NK, ep_k = ep_pt % NK, ep_E = E0 + ep_e;
            const bool ep_live = tid < NK * GG::TE * 6 && ep_E < d.ne;
            CT *ep_dst[2];
            CT old[2][EP_S];
#pragma unroll
            for (int rl = 0; rl < 2; ++rl) {
                const int r = EP_R * h + 2 * ep_rb + rl;
                ep_dst[rl] = S + (((size_t)ep_k * d.ne + (ep_live ? ep_E : 0)) * d.na + a) * kCh + r * 12 + EP_S * ep_sbk;
#pragma unroll
                for (int s = 0; s < EP_S; ++s) {
                    old[rl][s].x = 0;
                    old[rl][s].y = 0;
                    if (ep_live && !first_slot) old[rl][s] = ep_dst[rl][s];
                }
            }
            {
                const int qd = warp & 3, q = warp >> 2;
                const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (q ? kAccIm : 0u) + EP_COLS * h;
                float *vrow = sV + (q * kRowsMax + qd * 32 + lane) * EP_STRIDE;
#pragma unroll
                for (int c0 = 0; c0 < EP_COLS; c0 += 8) {
                    float v[8];
                    tmem_ld8(taddr + c0, v);
                    tmem_ld_wait();
                    tmem_pin(v);
#pragma unroll
                    for (int x = 0; x < 8; ++x) vrow[c0 + x] = v[x];
                }
            }
            __syncthreads();
            if (tid < NK * GG::TE * 6) {
                const int pt = ep_pt, rb = ep_rb, sbk = ep_sbk;
                const int e = ep_e, k = ep_k;
                float2 acc[2][EP_S];
#pragma unroll
                for (int rl = 0; rl < 2; ++rl)
#pragma unroll
                    for (int s = 0; s < EP_S; ++s) acc[rl][s] = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int m = GG::DA ? (k * 3 + j) * GG::DA_TE + e : pt * 3 + j;
                    const float *vre = sV + m * EP_STRIDE, *vim = sV + (kRowsMax + m) * EP_STRIDE;
#pragma unroll
                    for (int tt = 0; tt < 12; ++tt) {
                        float2 vv[2];
#pragma unroll
                        for (int rl = 0; rl < 2; ++rl) {
                            const int col = (2 * rb + rl) * 12 + tt;
                            vv[rl] = make_float2(vre[col], vim[col]);
                        }
#pragma unroll
                        for (int s = 0; s < EP_S; ++s) {
                            const float2 hv = sDh[j * kCh + (EP_S * sbk + s) * 12 + tt];
#pragma unroll
                            for (int rl = 0; rl < 2; ++rl) acc[rl][s] = cmul_conj_acc(acc[rl][s], vv[rl], hv);
                        }
                    }
                }
                if (ep_live && SSE_BC((ep_dst[0] - S) + EP_S - 1, (long long)d.nkz * d.ne * d.na * kCh, prm.status) &&
                    SSE_BC((ep_dst[1] - S) + EP_S - 1, (long long)d.nkz * d.ne * d.na * kCh, prm.status)) {
#pragma unroll
                    for (int rl = 0; rl < 2; ++rl)
#pragma unroll
                        for (int s = 0; s < EP_S; ++s) ep_dst[rl][s] = slot_sum<CT>(acc[rl][s], old[rl][s], first_slot);
                }
            }
            __syncthreads();
        }
        tc_fence_before();
        __syncthreads();
        if (*s_abort) {
            abort = true;
            abort_g = gg;
            abort_total = g_base + total;
            break;
        }
    }
    g_base += total;
    if (abort) break;
    }  // units

    // ---- teardown: nothing of ours may still be in flight when the CTA exits ----
    if (abort) {
        if (tid == 0) mma_commit(bar_fin);  // arrives once every MMA issued so far is done
        mbar_wait_bounded(bar_fin, 0, kWaitNs);
        // the bulk copies of the aborted stage and of the one prefetched after it
        if (abort_g >= 0) mbar_wait_bounded(&bar_g[abort_g & 1], (abort_g >> 1) & 1, kWaitNs);
        if (abort_g + 1 < abort_total)
            mbar_wait_bounded(&bar_g[(abort_g + 1) & 1], ((abort_g + 1) >> 1) & 1, kWaitNs);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---- the tensor-core form with the pre-product (Nkz = 5), warp-specialised ---------------
//
// Same arithmetic as the direct form above with X = dH_i . G taken from the tensor cores,
// but the CTA is split by role so that the MMAs of one stage run while the next ones are
// prepared.  Twelve builder warps: nine of them turn the pre-product X in TMEM into the main
// MMAs' B operand of each stage, all twelve run the epilogue of a job (the product with
// dH_j^dagger, also on the tensor cores: the builders re-encode the accumulators tile by
// tile as bf16 hi / lo and an MMA-issuing warp issues its MMAs).  Three MMA-issuing warps
// (lane 0 of each): one issues the MMAs into Re V and the post-product, one the MMAs into
// Im V, one the pre-product, so that one issuer's bookkeeping between stages hides behind the
// others' queued MMAs (an issuing thread blocks while the tensor pipe's queue is full, and its
// MMAs complete in its own issue order; the three write disjoint accumulators).  The first sits on
// the scheduler of the three builder warps without stage work (lane quarter 3: at Nkz = 5
// they add the previous job's staged post-product results into Sigma; below Nkz = 5 they
// are the encoders, and the Re-side issuer and the bulk-copy lane swap warps).  One bulk-copy warp streams the G
// slices into a ring and the slot tables into shared memory.  Hand-offs go through
// mbarriers: builders -> control "B of stage g built", "post-product tile built"; control
// -> builders through MMA commits ("X of a pair ready", "B buffer free", "job accumulated");
// the copies complete their own barriers.  The pre-product runs for two stages at once
// (N = 128: the two G slices side by side) as soon as the builders have read the previous
// pair (at its first stage), ahead of the main MMAs.
constexpr int kTcBuilders = 384;            // warps 0..11
constexpr int kTcXBuilders = 288;           // warps whose lane quarter holds X rows (warp % 4 < 3)
constexpr int kTcPrdWarp = 13;              // bulk copies
constexpr int kTcCtlWarp = 15;              // MMAs into Re V and the post-product
constexpr int kTcCtl2Warp = 14;             // MMAs into Im V
constexpr int kTcPreWarp = 12;              // the pre-product
constexpr int kTcThreads = 512;
constexpr int kTcRing = 2;   // pairs of G slices in flight
constexpr int kTcBStages = 2;  // B operands in flight: builders build stage g + 1 while the MMAs of stage g run
constexpr int kTcBStagesMax = 3;  // the encoding form takes a third where shared memory allows
constexpr uint32_t kTcPairBytes = 16384;  // one ring slot: two slices, [hi s0 | hi s1 | lo s0 | lo s1]
// TMEM columns of the warp-specialised kernel
constexpr uint32_t kTcAccIm = 160;             // Im V (Re V at 0), 144 columns each
constexpr uint32_t kTcPost0 = 320, kTcPost1 = 352;  // post-product accumulators, 32 columns each
constexpr uint32_t kTcPre = 384;               // X of a pair of stages, 2 x 64 columns
constexpr int kDhJ = 160;    // float2 per direction j of the padded dH copy
// Post-product Sigma_slot[(e, k), r, s] = sum_{j, t} V_j[(e, k)][r, t] conj(dH_j[s, t]) on the
// tensor cores: rows (r', e, k) of an M tile (three rows r per tile, four tiles; four rows
// and three tiles at Nkz <= 3), K = (j, t, re/im of V) = 72 padded to 80, N = (s, re/im of
// the product) = 24 padded to 32.
constexpr int kPostK = 80, kPostKc = kPostK / 8;            // K and its 16-byte chunks
constexpr uint32_t kPostSbo = kPostKc * 128;                // bytes between 8-row groups
constexpr uint32_t kPostAPlane = (kRowsMax / 8) * kPostSbo;  // 20480
constexpr uint32_t kPostBPlane = (32 / 8) * kPostSbo;        // 5120
constexpr int kTcBarBytes = 256;  // 24 mbarriers, the TMEM address and the flags; the unit index follows
constexpr int kTcEncoders = 96;   // encoding form: the warps of TMEM lane quarter 3 (3, 7, 11)
// Nkz = 5: the results of the job's last kStgTiles post-product tiles are staged in shared
// memory (rows of kStgStride floats: 24 values and padding against bank conflicts) and
// added to Sigma by the builder warps without stage work during the next job
constexpr int kStgTiles = 2, kStgStride = 28;

// dH_j[s, t] in shared memory: rows s in blocks of 4 with 4 float2 of padding between
// blocks, so the epilogue's three row blocks read distinct banks.
__device__ __forceinline__ int dh_at(int j, int s, int t) { return j * kDhJ + s * 12 + t + (s >> 2) * 4; }
// The epilogue's barrier among the warps that take part in it: all twelve builder warps, or
// in the encoding form the nine of lane quarters 0-2.
template <bool ENC>
__device__ __forceinline__ void builders_sync() {
    if constexpr (ENC) asm volatile("bar.sync 1, 288;" ::: "memory");
    else asm volatile("bar.sync 1, 384;" ::: "memory");
}

// Bytes of one slot's tables in the workspace: the direct Toeplitz table (rows w0 in
// [1 - TE, Nw + TE - 2]), the pre-product's dH operand and the post-product's conj(dH)
// operand, each in the shared-memory layout the MMAs read.
__host__ __device__ constexpr uint32_t tc_table_bytes(int nw) { return 2u * 2u * 16u * 2u * (uint32_t)(nw + 14) * 16u; }
__host__ __device__ constexpr uint32_t tc_entry_bytes(int nw) { return tc_table_bytes(nw) + 16384u + 2u * kPostBPlane; }

// Slot tables of one sign, one CTA per (atom a, slot b) with a neighbour: Dt folded over
// qz onto kz' = qz mod Nkz (T depends on (k - k') mod Nkz only), the direct table of the
// folded Dt, A_pre = the complex product dH_i . G as a real one (row re: (Re dH, -Im dH); row
// im: (Im dH, Re dH)), and B_post[(s, c'), (j, t, c)] for V conj(dH_j) = (Vr Hr + Vi Hi) +
// i (Vi Hr - Vr Hi); every value split into bf16 hi + lo.
template <int NK, typename CT>
__global__ void __launch_bounds__(256) sse_slot_tables_kernel(const CT *__restrict__ D, const CT *__restrict__ dH,
                                                              const int32_t *__restrict__ neigh,
                                                              const int32_t *__restrict__ rev, uint8_t *__restrict__ out,
                                                              int na, int nb, int nqz, int nw, int32_t *status) {
    using GG = Geo<NK>;
    extern __shared__ __align__(16) uint8_t tsm[];
    float2 *sDh = (float2 *)tsm;                      // [3][kDhJ] padded dH_j[s, t]
    float2 *dfold = (float2 *)(tsm + 3 * kDhJ * 8);   // [kappa][w][ij]
    const int a = blockIdx.x / nb, b = blockIdx.x % nb, tid = threadIdx.x;
    if (__ldg(neigh + (size_t)a * nb + b) < 0) return;
    const int da_rows = nw + 2 * GG::DA_TE - 2;
    uint8_t *tab = out + (size_t)blockIdx.x * tc_entry_bytes(nw);
    uint8_t *apre = tab + tc_table_bytes(nw), *bpost = apre + 16384;
    const CT *dh = dH + ((size_t)a * nb + b) * 3 * kCh;
    for (int x = tid; x < 3 * kCh; x += 256) sDh[dh_at(x / kCh, (x % kCh) / 12, x % 12)] = load_c32(dh + x);
    for (int x = tid; x < NK * nw * 9; x += 256) {
        const int ij = x % 9, w = (x / 9) % nw, kap = x / (9 * nw);
        float2 acc = make_float2(0.f, 0.f);
        for (int q = kap; q < nqz; q += NK) {
            const float2 v = load_dt(D, neigh, rev, q, w, nw, na, nb, a, b, ij, status);
            acc.x += v.x;
            acc.y += v.y;
        }
        dfold[x] = acc;
    }
    __syncthreads();
    // direct table: [q = Re, Im][hi, lo][group (k, j)][K group][row r] x 16 bytes, entry
    // (i, k') of row r = Re or Im of Df_ij[(k - k') mod Nkz][r - (TE - 1)]; at Nkz <= 3
    // [q][group][K group 0..3][row r] with the split products in K: (hi | hi | lo) of the entries
    if constexpr (NK <= 3) {
        constexpr int L = 3 * NK;
        const int nrow = 2 * GG::DA_GROUPS * da_rows;
        for (int x = tid; x < nrow; x += 256) {
            const int r = x % da_rows, gq = (x / da_rows) % GG::DA_GROUPS, q = x / (da_rows * GG::DA_GROUPS);
            const int k = gq / 3, j = gq % 3, w0 = r - (GG::DA_TE - 1);
            float v[L];
#pragma unroll
            for (int kk = 0; kk < L; ++kk) {
                float val = 0.f;
                if (gq < 3 * NK && w0 >= 0 && w0 < nw) {
                    const int i = kk / NK, kp = kk % NK;
                    const float2 T = dfold[(((k - kp + NK) % NK) * nw + w0) * 9 + i * 3 + j];
                    val = q ? T.y : T.x;
                }
                v[kk] = val;
            }
            uint32_t wv[16];
            splitk_row<L>(v, true, wv);
#pragma unroll
            for (int kg = 0; kg < 4; ++kg)
                *(uint4 *)(tab + ((((size_t)q * GG::DA_GROUPS + gq) * 4 + kg) * da_rows + r) * 16) =
                    make_uint4(wv[4 * kg], wv[4 * kg + 1], wv[4 * kg + 2], wv[4 * kg + 3]);
        }
    }
    const int nitems = NK <= 3 ? 0 : 2 * GG::DA_GROUPS * 2 * da_rows;
    for (int x = tid; x < nitems; x += 256) {
        const int r = x % da_rows, kg = (x / da_rows) % 2, gq = (x / (2 * da_rows)) % GG::DA_GROUPS;
        const int q = x / (2 * da_rows * GG::DA_GROUPS);
        const int k = gq / 3, j = gq % 3, w0 = r - (GG::DA_TE - 1);
        float v[8];
#pragma unroll
        for (int xx = 0; xx < 8; ++xx) {
            const int kk = kg * 8 + xx;
            float val = 0.f;
            if (gq < 3 * NK && kk < 3 * NK && w0 >= 0 && w0 < nw) {
                const int i = kk / NK, kp = kk % NK;
                const float2 T = dfold[(((k - kp + NK) % NK) * nw + w0) * 9 + i * 3 + j];
                val = q ? T.y : T.x;
            }
            v[xx] = val;
        }
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) {
            const uint2 hl = split2_bf16(v[2 * xx], v[2 * xx + 1]);
            hv[xx] = hl.x;
            lv[xx] = hl.y;
        }
        const size_t base_hi = ((((size_t)(q * 2 + 0) * GG::DA_GROUPS + gq) * 2 + kg) * da_rows + r) * 16;
        const size_t base_lo = ((((size_t)(q * 2 + 1) * GG::DA_GROUPS + gq) * 2 + kg) * da_rows + r) * 16;
        *(uint4 *)(tab + base_hi) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *(uint4 *)(tab + base_lo) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    // A_pre row m = 32 (r / 4) + 8 i + 4 (re/im) + r % 4 (lanes 24..31 of each quarter and
    // the last quarter zero): one TMEM lane quarter holds every i for four r
    for (int x = tid; x < kRowsMax * 4; x += 256) {
        const int m = x >> 2, kg = x & 3;
        const int mq = m >> 5, i = (m >> 3) & 3, pr = (m >> 2) & 1, r = 4 * mq + (m & 3);
        float v[8];
#pragma unroll
        for (int xx = 0; xx < 8; ++xx) {
            const int kk = kg * 8 + xx;
            float val = 0.f;
            if (mq < 3 && i < 3 && kk < 24) {
                const int pc = kk / 12, u = kk % 12;
                const float2 h = sDh[dh_at(i, r, u)];
                val = pr ? (pc ? h.x : h.y) : (pc ? -h.y : h.x);
            }
            v[xx] = val;
        }
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) {
            const uint2 hl = split2_bf16(v[2 * xx], v[2 * xx + 1]);
            hv[xx] = hl.x;
            lv[xx] = hl.y;
        }
        uint8_t *dst = apre + (m >> 3) * 512 + kg * 128 + (m & 7) * 16;
        *(uint4 *)dst = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *(uint4 *)(dst + 8192) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    for (int x = tid; x < 32 * kPostKc; x += 256) {
        const int row = x / kPostKc, kc = x % kPostKc, s2 = row >> 1, cp = row & 1;
        float v[8];
#pragma unroll
        for (int xx = 0; xx < 8; ++xx) {
            const int kk = kc * 8 + xx;
            float val = 0.f;
            if (row < 24 && kk < 72) {
                const int j = kk / 24, t = (kk % 24) >> 1, c = kk & 1;
                const float2 h = sDh[dh_at(j, s2, t)];
                val = cp ? (c ? h.x : -h.y) : (c ? h.y : h.x);
            }
            v[xx] = val;
        }
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) {
            const uint2 hl = split2_bf16(v[2 * xx], v[2 * xx + 1]);
            hv[xx] = hl.x;
            lv[xx] = hl.y;
        }
        uint8_t *dst = bpost + (row >> 3) * kPostSbo + kc * 128 + (row & 7) * 16;
        *(uint4 *)dst = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *(uint4 *)(dst + kPostBPlane) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
}

template <int NK, typename CT, bool ENC, int BST>
__global__ void __launch_bounds__(kTcThreads, 1) sse_tc_kernel(const __grid_constant__ MixParams prm) {
    using GG = Geo<NK>;
    constexpr int TE = GG::DA_TE;        // energies per tile of this form (rows (k, j, e): 3 NK TE)
    constexpr int kVRows = 3 * NK * TE;  // accumulator rows used
    // post-product tiles: rows (r', e, k) for kRpt rows r of the block (four at Nkz <= 3,
    // where 4 TE Nkz <= 96 rows still leave lane quarter 3 to the encoders), kPT per job
    constexpr int kRpt = NK <= 3 ? 4 : 3;
    constexpr int kPT = 12 / kRpt;
    constexpr int kPostRows = kRpt * TE * NK;
    static_assert(kVRows <= kRowsMax && kPostRows <= kRowsMax, "tile rows");
    // The encoding form (ENC) copies raw G blocks and has the warps of TMEM lane quarter 3
    // encode them for the pre-product; it needs every accumulator and post-product row in
    // lane quarters 0-2, so that those warps never take part in the epilogue.
    static_assert(!ENC || (kVRows <= 96 && kPostRows <= 96), "encoding form: rows in lane quarters 0-2");
    // At Nkz <= 3 the split products are folded into K (K row (i, k') = 3 Nkz <= 9 values):
    // B planes [Re X, Im X] of K = 32 and two MMAs per complex term instead of three.
    constexpr bool SPLITK = NK <= 3;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Roles.  The encoding form's encoders are the warps of lane quarter 3, which share SM
    // sub-partition 3 (warp % 4) with warp 15; there the Re-side issuer moves to warp 13 and
    // the (light) bulk-copy lane to warp 15, so that no issuer shares a scheduler with them.
    constexpr int kCtlWarp = ENC ? kTcPrdWarp : kTcCtlWarp, kPrdWarp = ENC ? kTcCtlWarp : kTcPrdWarp;
    const bool ctl = warp == kCtlWarp || warp == kTcCtl2Warp || warp == kTcPreWarp;  // MMA-issuing warps
    const bool re_side = warp == kCtlWarp;     // main MMAs into Re V, the post-product
    const bool im_side = warp == kTcCtl2Warp;  // main MMAs into Im V
    const bool pre_side = warp == kTcPreWarp;  // the pre-product
    const bool prd = warp == kPrdWarp;         // bulk-copy warp
    const int nw = prm.nw;
    const int omega_max = prm.omega_first + nw - 1;
    const int da_rows = nw + 2 * GG::DA_TE - 2;

    uint8_t *sB = smem + prm.off_b;              // [2 stages][re hi, re lo, im hi, im lo]
    uint8_t *sApost = smem + prm.off_b;          // epilogue: post-product A tile over the B stages
    uint8_t *sBpost = smem + prm.off_bp;         // post-product B of the slot: conj(dH_j) [hi, lo]
    uint8_t *sRing = smem + prm.off_g;           // [kTcRing] pairs of re-encoded G slices
    uint8_t *sRaw = smem + prm.off_x;            // encoding form: [kTcRing] pairs of raw G blocks
    uint8_t *sApre = smem + prm.off_a;           // pre-product A: dH operand [hi, lo]
    uint8_t *sTab = smem + prm.off_df;           // direct Toeplitz table of the slot
    float *stg = (!ENC && prm.off_stg) ? (float *)(smem + prm.off_stg) : nullptr;  // [kStgTiles][kPostRows][kStgStride]
    uint64_t *bars = (uint64_t *)(smem + prm.off_bar);
    uint64_t *bar_g = bars;                          // [kTcRing] pair of slices landed
    uint64_t *bar_empty = bar_g + kTcRing;           // [kTcRing] pre-product done with a ring slot
    uint64_t *bar_bready = bar_empty + kTcRing;      // [nbst] B of a stage built
    uint64_t *bar_mma = bar_bready + kTcBStagesMax;  // [nbst] main MMAs of a stage done (B free)
    uint64_t *bar_post = bar_mma + kTcBStagesMax;    // [2] post-product MMAs of a tile done
    uint64_t *bar_pre = bar_post + 2;                // pre-product of a pair done
    uint64_t *bar_job = bar_pre + 1;                 // last MMAs of a job done
    uint64_t *bar_slot = bar_job + 1;                // the slot's pre- and post-product operands copied in
    uint64_t *bar_fin = bar_slot + 1;                // abort: every MMA issued so far done
    uint64_t *bar_apost = bar_fin + 1;               // post-product A tile built
    uint64_t *bar_slotfree = bar_apost + 1;          // every MMA of the previous slot done
    uint64_t *bar_tab = bar_slotfree + 1;            // the slot's direct table copied in
    uint64_t *bar_enc = bar_tab + 1;                 // [kTcRing] encoding form: a pair encoded into the ring
    uint64_t *bar_rawfree = bar_enc + kTcRing;       // [kTcRing] encoding form: a raw pair consumed
    uint64_t *bar_xfree = bar_rawfree + kTcRing;     // the builders have read X of a pair (TMEM free)
    uint32_t *s_tmem = (uint32_t *)(bar_xfree + 1);
    static_assert((4 * kTcRing + 2 * kTcBStagesMax + 10) * 8 + 7 * 4 <= kTcBarBytes, "barrier area");
    constexpr int nbst = BST;  // B buffers in flight (2, or 3 in the encoding form where they fit)
    // abort flags, each written only by its role (builders: s_abort[0]) before the unit's
    // closing barrier and read by every thread after it
    int *s_abort = (int *)(s_tmem + 1);          // [2]
    int *s_abort_ctl = s_abort + 2;
    int *s_nvalid = s_abort + 3;
    int *s_abort_prd = s_abort + 4;
    int *s_abort_enc = s_abort + 5;
    long long *s_unit = (long long *)(smem + prm.off_bar + kTcBarBytes);
    int *s_slot = (int *)(s_unit + 1);
    int *s_f = s_slot + kMaxSlots;

    if (tid == 0) {
        for (int b = 0; b < kTcRing; ++b) mbar_init(&bar_g[b], 1);
        mbar_init(bar_pre, 1);
        for (int b = 0; b < nbst; ++b) {
            mbar_init(&bar_bready[b], kTcXBuilders);
            mbar_init(&bar_mma[b], 2);  // a commit from each issuing warp
        }
        mbar_init(bar_job, 2);       // both issuing warps
        mbar_init(bar_slot, 1);
        mbar_init(bar_tab, 1);
        mbar_init(bar_slotfree, 3);  // the three issuing warps
        mbar_init(bar_fin, 3);       // the three issuing warps
        mbar_init(bar_apost, ENC ? kTcBuilders - kTcEncoders : kTcBuilders);
        mbar_init(bar_xfree, kTcXBuilders);
        mbar_init(&bar_post[0], 1);
        mbar_init(&bar_post[1], 1);
        for (int b = 0; b < kTcRing; ++b) {
            mbar_init(&bar_empty[b], 1);
            mbar_init(&bar_enc[b], kTcEncoders);
            mbar_init(&bar_rawfree[b], kTcEncoders);
        }
        fence_mbar_init();
        s_abort[0] = 0;
        s_abort[1] = 0;
        *s_abort_ctl = 0;
        *s_abort_prd = 0;
        *s_abort_enc = 0;
    }
    if (warp == 0) {
        tmem_alloc(s_tmem, kTmemCols);
        tmem_relinquish();
    }
    if (ENC && (warp & 3) == 3 && warp < kTcBuilders / 32) {
        // the encoders write only the live part of the ring's slices (rows below 12 Nkz, K below
        // 24); the rest stays zero from here on
        for (int x = (warp >> 2) * 32 + lane; x < kTcRing * kTcPairBytes / 16; x += kTcEncoders)
            *(uint4 *)(sRing + (size_t)x * 16) = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    int last_g[kTcRing];  // bulk-copy lane 0: last pair copied into each ring slot
    int slot_cp = 0;      // bulk-copy lane 0: slot tables copied so far
    int pair_ctr = 0;     // pairs of stages so far (each role keeps its own count)
#pragma unroll
    for (int b = 0; b < kTcRing; ++b) last_g[b] = -1;
    int g_base = 0, job_ctr = 0, slot_ctr = 0;
    int tile_ctr = 0;  // post-product tiles so far (phases of bar_apost / bar_post)
    bool abort = false;
    for (long long iter = 0;; ++iter) {
        __syncthreads();
        if (tid == 0) {
            long long u;
            if (prm.queue) u = atomicAdd(prm.queue, 1);
            else u = iter == 0 ? (long long)blockIdx.x : prm.total_units;
            if (*(volatile int32_t *)prm.status != 0) u = prm.total_units;
            *s_unit = u;
        }
        __syncthreads();
        const long long unit = *s_unit;
        if (unit >= prm.total_units) break;
        int ii = 0;
        while (ii + 1 < prm.n_inst && prm.inst[ii + 1].unit_begin <= unit) ++ii;
        const InstDesc &I = prm.inst[ii];
        const long long local = unit - I.unit_begin;
        const int sign = (int)(local / ((long long)I.na * I.nchunks));
        const long long rem = local - (long long)sign * I.na * I.nchunks;
        const int a = (int)(rem / I.nchunks), chunk = (int)(rem % I.nchunks);
        const Dims d{prm.nkz, I.nqz, I.ne, nw, I.na, I.nb, prm.omega_first};
        CT *__restrict__ S = (CT *)I.S[sign];
        const int t_begin = chunk * I.tiles_per_cta;
        const int t_end = min(I.ntiles, t_begin + I.tiles_per_cta);
        if (tid == 0) {
            int nv = 0;
            for (int b = 0; b < d.nb && nv < kMaxSlots; ++b) {
                const int f = __ldg(I.neigh + (size_t)a * d.nb + b);
                if (f >= 0) {
                    s_slot[nv] = b;
                    s_f[nv] = f;
                    ++nv;
                }
            }
            *s_nvalid = nv;
        }
        __syncthreads();
        const int nvalid = *s_nvalid;
        const int total = (t_end - t_begin) * nvalid * prm.nst;
        if (nvalid == 0) {
            for (int t = t_begin; t < t_end; ++t)
                for (int x = tid; x < NK * TE * kCh; x += kTcThreads) {
                    const int e = x / (NK * kCh), k = (x / kCh) % NK, c = x % kCh;
                    const int E = t * TE + e;
                    const size_t idx = (((size_t)k * d.ne + E) * d.na + a) * kCh + c;
                    if (E < d.ne && SSE_BC(idx, (long long)d.nkz * d.ne * d.na * kCh, prm.status)) {
                        CT z;
                        z.x = 0;
                        z.y = 0;
                        S[idx] = z;
                    }
                }
        }
        // stage position (tile, valid-slot index, stage within the job), slot-major
        struct Pos {
            int t, vs, st;
        };
        auto advance = [&](Pos &p) {
            if (++p.st < prm.nst) return;
            p.st = 0;
            if (++p.t == t_end) {
                p.t = t_begin;
                ++p.vs;
            }
        };

        if (ctl) {
            // ========== MMA-issuing warps (lane 0): Re side, Im side, pre-product side ==========
            if (lane == 0) {
                // descriptors: fixed parts built once; a shift of the start address is an add
                // on the descriptor's low field (shared addresses stay below 2^18)
                const uint64_t pa_h0 = smem_desc(smem_u32(sApre), 128, 512), pa_l0 = smem_desc(smem_u32(sApre) + 8192, 128, 512);
                const uint64_t pb_h0 = smem_desc(smem_u32(sRing), 128, 512), pb_l0 = smem_desc(smem_u32(sRing) + 8192, 128, 512);
                // pre-product of the next pair of stages: rows (r / 4, i, re/im, r % 4), N = (stage
                // of the pair, t / 4, k', t % 4) = 128, K = (re/im of G, u)
                auto premma = [&]() -> bool {
                    const int slot = pair_ctr % kTcRing;
                    // the pair of slices: copied in (stored form) or encoded by the encoder warps
                    if (!mbar_wait_bounded(ENC ? &bar_enc[slot] : &bar_g[slot], (pair_ctr / kTcRing) & 1, kWaitNs))
                        return false;
                    tc_fence_after();
                    constexpr uint32_t idesc_x = idesc_bf16_f32(kRowsMax, 128);
                    const uint64_t boff = (uint64_t)((slot * kTcPairBytes) >> 4);
                    const uint32_t dx = tmem + kTcPre;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ko = (uint64_t)(ks * 256 >> 4);
                        mma_ss(dx, pa_h0 + ko, pb_h0 + boff + ko, idesc_x, ks ? 1u : 0u);
                        mma_ss(dx, pa_h0 + ko, pb_l0 + boff + ko, idesc_x, 1u);
                        mma_ss(dx, pa_l0 + ko, pb_h0 + boff + ko, idesc_x, 1u);
                    }
                    mma_commit(bar_pre);
                    mma_commit(&bar_empty[slot]);  // the ring slot can be refilled
                    ++pair_ctr;
                    return true;
                };
                Pos m{t_begin, 0, 0};
                constexpr uint32_t idesc = idesc_bf16_f32(kRowsMax, kCh);
                constexpr uint32_t idesc_negb = idesc | (1u << 14);
                const uint32_t lbo_a = (uint32_t)da_rows * 16, sbo_a = (SPLITK ? 4u : 2u) * lbo_a;
                const uint32_t tstride = (uint32_t)GG::DA_GROUPS * 2 * da_rows * 16;
                // A (direct table) at row 0 for (re/im, hi/lo); stage st starts at row nw - 1 - st + TE - 1
                // (split-in-K form: ta[0] = the Re table, ta[2] = the Im table, two K chunks each)
                uint64_t ta[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) ta[x] = smem_desc(smem_u32(sTab) + (uint32_t)x * tstride, lbo_a, sbo_a);
                // B (X of the stage) of B stage 0; stage 1 is kBufStep further, planes kPlaneStep apart
                const uint64_t tb0 = smem_desc(smem_u32(sB), 128, SPLITK ? 2 * GG::DA_SBO_B : GG::DA_SBO_B);
                constexpr uint64_t kPlaneStep = GG::DA_B_PLANE >> 4, kBufStep = (4 * GG::DA_B_PLANE) >> 4;
                const uint64_t pp_ah = smem_desc(smem_u32(sApost), 128, kPostSbo);
                const uint64_t pp_al = smem_desc(smem_u32(sApost) + kPostAPlane, 128, kPostSbo);
                const uint64_t pp_bh = smem_desc(smem_u32(sBpost), 128, kPostSbo);
                const uint64_t pp_bl = smem_desc(smem_u32(sBpost) + kPostBPlane, 128, kPostSbo);
                const int slot_len = (t_end - t_begin) * prm.nst;  // stages of one slot in this unit
                bool ok = true;
                if (pre_side) {
                    // the pre-product, pair by pair: the next pair's X goes into TMEM as soon as
                    // the builders have read the previous one, ahead of the stages that use it
                    const int npairs = (slot_len + 1) / 2;
                    for (int vs = 0; vs < nvalid && ok; ++vs) {
                        // the slot's pre-product operand copied in
                        if (!(ok = mbar_wait_bounded(bar_slot, slot_ctr & 1, kWaitNs))) break;
                        ++slot_ctr;
                        tc_fence_after();
                        for (int pr = 0; pr < npairs && ok; ++pr) {
                            if (pair_ctr > 0 && !(ok = mbar_wait_bounded(bar_xfree, (pair_ctr - 1) & 1, kWaitNs))) break;
                            tc_fence_after();
                            ok = premma();
                        }
                        if (ok) mma_commit(bar_slotfree);  // its pre-products of the slot
                    }
                }
                int o = 0;  // stage index within the slot
                for (int g = 0; g < (pre_side ? 0 : total); ++g, advance(m), o = (o + 1 == slot_len) ? 0 : o + 1) {
                    const int gg = g_base + g;
                    const bool job_first = m.st == 0, job_last = m.st == prm.nst - 1;
                    const int slot_rem = slot_len - 1 - o;  // stages after this one in its slot
                    if (o == 0 && re_side) {
                        // the slot's post-product operand
                        if (!(ok = mbar_wait_bounded(bar_slot, slot_ctr & 1, kWaitNs))) break;
                        tc_fence_after();
                    }
                    const int bb = gg % nbst, use = gg / nbst;  // B buffer and its use count
                    if (!(ok = mbar_wait_bounded(&bar_bready[bb], use & 1, kWaitNs))) break;
                    if (o == 0) {
                        ok = mbar_wait_bounded(bar_tab, slot_ctr & 1, kWaitNs);
                        ++slot_ctr;
                        if (!ok) break;
                    }
                    tc_fence_after();
                    const uint64_t r_start = (uint64_t)(nw - 1 - m.st + GG::DA_TE - 1);
                    const uint64_t are_h = ta[0] + r_start, are_l = ta[1] + r_start;
                    const uint64_t aim_h = ta[2] + r_start, aim_l = ta[3] + r_start;
                    const uint64_t b0 = tb0 + (uint64_t)bb * kBufStep;
                    const uint64_t bre_h = b0, bre_l = b0 + kPlaneStep, bim_h = b0 + 2 * kPlaneStep, bim_l = b0 + 3 * kPlaneStep;
                    const uint32_t dre = tmem, dim = tmem + kTcAccIm;
                    const uint32_t acc0 = job_first ? 0u : 1u;
                    if constexpr (SPLITK) {
                        // planes [Re X | Im X] (K = 32 each) and tables [Re T | Im T] (K = 32 each)
                        const uint64_t a_k1 = (uint64_t)((2u * lbo_a) >> 4), b_k1 = 256 >> 4;
                        const uint64_t br = b0, bi = b0 + 2 * kPlaneStep;
                        if (re_side) {
                            // Re V = Re T Re X - Im T Im X
                            mma_ss(dre, are_h, br, idesc, acc0);
                            mma_ss(dre, are_h + a_k1, br + b_k1, idesc, 1u);
                            mma_ss(dre, aim_h, bi, idesc_negb, 1u);
                            mma_ss(dre, aim_h + a_k1, bi + b_k1, idesc_negb, 1u);
                        } else {
                            // Im V = Im T Re X + Re T Im X
                            mma_ss(dim, aim_h, br, idesc, acc0);
                            mma_ss(dim, aim_h + a_k1, br + b_k1, idesc, 1u);
                            mma_ss(dim, are_h, bi, idesc, 1u);
                            mma_ss(dim, are_h + a_k1, bi + b_k1, idesc, 1u);
                        }
                    } else if (re_side) {
                        // Re V = Re T Re X - Im T Im X
                        mma_ss(dre, are_h, bre_h, idesc, acc0);
                        mma_ss(dre, are_h, bre_l, idesc, 1u);
                        mma_ss(dre, are_l, bre_h, idesc, 1u);
                        mma_ss(dre, aim_h, bim_h, idesc_negb, 1u);
                        mma_ss(dre, aim_h, bim_l, idesc_negb, 1u);
                        mma_ss(dre, aim_l, bim_h, idesc_negb, 1u);
                    } else {
                        // Im V = Im T Re X + Re T Im X
                        mma_ss(dim, aim_h, bre_h, idesc, acc0);
                        mma_ss(dim, aim_h, bre_l, idesc, 1u);
                        mma_ss(dim, aim_l, bre_h, idesc, 1u);
                        mma_ss(dim, are_h, bim_h, idesc, 1u);
                        mma_ss(dim, are_h, bim_l, idesc, 1u);
                        mma_ss(dim, are_l, bim_h, idesc, 1u);
                    }
                    mma_commit(&bar_mma[bb]);
                    if (job_last && im_side) {
                        mma_commit(bar_job);
                        if (slot_rem == 0) mma_commit(bar_slotfree);
                    }
                    if (job_last && re_side) {
                        mma_commit(bar_job);
                        // post-product of the job, one M tile at a time as the builders fill it
                        constexpr uint32_t idesc_p = idesc_bf16_f32(kRowsMax, 32);
                        for (int q = 0; q < kPT && ok; ++q, ++tile_ctr) {
                            if (!(ok = mbar_wait_bounded(bar_apost, tile_ctr & 1, kWaitNs))) break;
                            tc_fence_after();
                            const uint32_t dp = tmem + ((tile_ctr & 1) ? kTcPost1 : kTcPost0);
#pragma unroll
                            for (int ks = 0; ks < kPostK / 16; ++ks) {
                                const uint64_t ko = (uint64_t)(ks * 256 >> 4);
                                mma_ss(dp, pp_ah + ko, pp_bh + ko, idesc_p, ks ? 1u : 0u);
                                mma_ss(dp, pp_ah + ko, pp_bl + ko, idesc_p, 1u);
                                mma_ss(dp, pp_al + ko, pp_bh + ko, idesc_p, 1u);
                            }
                            mma_commit(&bar_post[tile_ctr & 1]);
                        }
                        if (!ok) break;
                        if (slot_rem == 0) mma_commit(bar_slotfree);  // the slot's tables can be replaced
                    }
                }
                if (!ok) {
                    *s_abort_ctl = 1;
                    atomicOr(prm.status, kStatusTimeout);
                }
            }
            __syncwarp();
        } else if (prd) {
            // ================= bulk-copy warp: G slices into the ring (lane 0) =================
            if (lane == 0) {
                const uint8_t *gws = I.gws[sign];
                const uint32_t tbytes = tc_table_bytes(nw), ebytes = tc_entry_bytes(nw);
                const int slot_len = (t_end - t_begin) * prm.nst;
                const long long zero = (long long)d.ne * d.na;  // the zero slice
                bool ok = true;
                // one pair of slices (stage offsets o, o + 1 of the slot) into the next ring slot;
                // the encoding form copies the pair's raw G blocks instead, [h][k'][144] values
                auto issue_pair = [&](int o, int f) -> bool {
                    const int slot = pair_ctr % kTcRing, use = pair_ctr / kTcRing;
                    if constexpr (ENC) {
                        // raw slot free: the encoders are done with its previous pair (first use: free)
                        if (!mbar_wait_bounded(&bar_rawfree[slot], (use & 1) ^ 1, kWaitNs)) return false;
                        const CT *G = (const CT *)I.G[sign];
                        uint32_t bytes = 0;
                        int Eps[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            Eps[h] = -1;
                            if (o + h < slot_len) {
                                const int t = t_begin + (o + h) / prm.nst, st = (o + h) % prm.nst;
                                const int Ep = t * TE - omega_max + st;
                                if (Ep >= 0 && Ep < d.ne) Eps[h] = Ep;
                            }
                            if (Eps[h] >= 0) bytes += NK * kCh * (uint32_t)sizeof(CT);
                        }
                        mbar_arrive_expect_tx(&bar_g[slot], bytes);  // no bytes: completes at once
                        uint8_t *dst = sRaw + (size_t)slot * 2 * NK * kCh * sizeof(CT);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (Eps[h] < 0) continue;
                            for (int kp = 0; kp < NK; ++kp) {
                                const size_t src = (((size_t)kp * d.ne + Eps[h]) * d.na + f) * kCh;
                                if (SSE_BC(src + kCh - 1, (long long)d.nkz * d.ne * d.na * kCh, prm.status))
                                    bulk_g2s(dst + (h * NK + kp) * kCh * sizeof(CT), G + src, kCh * (uint32_t)sizeof(CT),
                                             &bar_g[slot]);
                            }
                        }
                        last_g[slot] = pair_ctr++;
                        return true;
                    }
                    // ring slot free: the pre-product of its previous pair is done (first use: free)
                    if (!mbar_wait_bounded(&bar_empty[slot], (use & 1) ^ 1, kWaitNs)) return false;
                    mbar_arrive_expect_tx(&bar_g[slot], kTcPairBytes);
                    uint8_t *dst = sRing + slot * kTcPairBytes;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // the zero slice stands in for energies below or above the grid and for
                        // the missing second stage of an odd-length slot
                        long long slice = zero;
                        if (o + h < slot_len) {
                            const int t = t_begin + (o + h) / prm.nst, st = (o + h) % prm.nst;
                            const int Ep = t * TE - omega_max + st;
                            if (Ep >= 0 && Ep < d.ne) slice = (long long)Ep * d.na + f;
                        }
                        const uint8_t *sl = gws + slice * kXpSlice;
                        // a skipped copy leaves the pair's barrier short: its wait then times out
                        if (SSE_BC(slice, (long long)d.ne * d.na + 1, prm.status)) {
                            bulk_g2s(dst + h * 4096, sl, 4096, &bar_g[slot]);
                            bulk_g2s(dst + 8192 + h * 4096, sl + 4096, 4096, &bar_g[slot]);
                        }
                    }
                    last_g[slot] = pair_ctr++;
                    return true;
                };
                const int npairs = (slot_len + 1) / 2;
                for (int vs = 0; vs < nvalid && ok; ++vs) {
                    const int f = s_f[vs];
                    // the slot's first pairs go ahead of its tables: they only need free ring slots
                    int pr = 0;
                    for (; pr < npairs && pr < kTcRing && ok; ++pr) ok = issue_pair(2 * pr, f);
                    if (!ok) break;
                    // its tables replace the previous slot's once every MMA that read those is
                    // done (the CTA's first slot: nothing to wait for)
                    if (!(ok = mbar_wait_bounded(bar_slotfree, (slot_cp & 1) ^ 1, kWaitNs))) break;
                    // the small operands first: the pre-product can start while the table streams in
                    // (the failure-injection hook skips the tables of the CTA's first unit's second
                    // slot, its only slot if it has one)
                    if (!(prm.inject && iter == 0 && vs == (nvalid > 1 ? 1 : 0)) &&
                        SSE_BC((size_t)a * d.nb + s_slot[vs], (long long)d.na * d.nb, prm.status)) {
                        const uint8_t *src = I.sws[sign] + ((size_t)a * d.nb + s_slot[vs]) * ebytes;
                        mbar_arrive_expect_tx(bar_slot, 16384 + 2 * kPostBPlane);
                        bulk_g2s(sApre, src + tbytes, 16384, bar_slot);
                        bulk_g2s(sBpost, src + tbytes + 16384, 2 * kPostBPlane, bar_slot);
                        mbar_arrive_expect_tx(bar_tab, tbytes);
                        bulk_g2s(sTab, src, tbytes, bar_tab);
                        ++slot_cp;
                    }
                    for (; pr < npairs && ok; ++pr) ok = issue_pair(2 * pr, f);
                }
                if (!ok) {
                    *s_abort_prd = 1;
                    atomicOr(prm.status, kStatusTimeout);
                }
            }
            __syncwarp();
        } else if (ENC && (warp & 3) == 3 && warp < kTcBuilders / 32) {
            // ================= encoder warps (encoding form): raw G -> pre-product operand =================
            // Per pair of stages, in the order the bulk-copy warp copies them: wait for the raw
            // blocks and for the ring slot's previous pre-product, then write the slices -- rows
            // n' = (t / 4) 4 Nkz + k' 4 + t % 4 (12 Nkz used of 64), K = (re/im of G, u) (24 of
            // 32), bf16 hi then lo plane, core-matrix order -- and hand the slot to the pre-product.
            // One thread per live row (stage h, n'): the row's K values are the column t of the
            // block G[k'] (twelve u, re then im).
            const int et = (warp >> 2) * 32 + lane;  // 0 .. 95
            const int slot_len = (t_end - t_begin) * prm.nst;
            const int npairs = (slot_len + 1) / 2;
            bool ok = true;
            for (int vs = 0; vs < nvalid && ok; ++vs)
                for (int pr = 0; pr < npairs && ok; ++pr, ++pair_ctr) {
                    const int slot = pair_ctr % kTcRing, use = pair_ctr / kTcRing;
                    if (!(ok = mbar_wait_bounded(&bar_g[slot], use & 1, kWaitNs))) break;
                    if (!(ok = mbar_wait_bounded(&bar_empty[slot], (use & 1) ^ 1, kWaitNs))) break;
                    const uint8_t *raw = sRaw + (size_t)slot * 2 * NK * kCh * sizeof(CT);
                    uint8_t *dst = sRing + slot * kTcPairBytes;
                    for (int it = et; it < 2 * 12 * NK; it += kTcEncoders) {  // (stage h, live row n')
                        const int h = it / (12 * NK), np = it % (12 * NK);
                        const int o2 = 2 * pr + h;
                        bool live = o2 < slot_len;
                        if (live) {
                            const int t = t_begin + o2 / prm.nst, st = o2 % prm.nst;
                            const int Ep = t * TE - omega_max + st;
                            live = Ep >= 0 && Ep < d.ne;
                        }
                        const int blk = np / (4 * NK), kp = (np % (4 * NK)) / 4, t = 4 * blk + np % 4;
                        const CT *col = (const CT *)raw + (h * NK + kp) * kCh + t;
                        float v[24];  // K = u (re), 12 + u (im)
#pragma unroll
                        for (int u = 0; u < 12; ++u) {
                            const float2 c = live ? load_c32_smem(col + u * 12) : make_float2(0.f, 0.f);
                            v[u] = c.x;
                            v[12 + u] = c.y;
                        }
                        uint8_t *pd = dst + h * 4096 + (np >> 3) * 512 + (np & 7) * 16;
#pragma unroll
                        for (int kg = 0; kg < 3; ++kg) {
                            uint32_t hv[4], lv[4];
#pragma unroll
                            for (int xx = 0; xx < 4; ++xx) {
                                const uint2 hl = split2_bf16(v[8 * kg + 2 * xx], v[8 * kg + 2 * xx + 1]);
                                hv[xx] = hl.x;
                                lv[xx] = hl.y;
                            }
                            *(uint4 *)(pd + kg * 128) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                            *(uint4 *)(pd + 8192 + kg * 128) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                        }
                    }
                    fence_proxy_async_smem();
                    mbar_arrive(&bar_rawfree[slot]);
                    mbar_arrive(&bar_enc[slot]);
                }
            if (!ok) {
                if (lane == 0) *s_abort_enc = 1;
                atomicOr(prm.status, kStatusTimeout);
            }
        } else if (warp < kTcBuilders / 32) {
            // ================= builder warps =================
            Pos cur{t_begin, 0, 0};
            const int slot_len = (t_end - t_begin) * prm.nst;
            int o = 0;                // stage index within the slot
            uint32_t xnext[3 * NK];   // X warps: K row of the pair's second stage, kept until then
            const int q4 = warp & 3, cb = warp >> 2;
            const bool xw = q4 < 3;  // warps whose lane quarter holds X rows
            // A failed wait marks this builder bad and skips its later waits; builders never
            // leave the loop early, so every one reaches each builders_sync.
            bool bad = false;
            // Staged results of the previous job (Nkz = 5): its last kStgTiles post-product
            // tiles, added to Sigma by the three warps without stage work (lane quarter 3)
            // while this job runs.  Element (tile, row, s) always goes to the same thread, so
            // the first slot's store and later slots' reductions to an address are ordered.
            bool pend = false, pend_first = false;
            int pend_E0 = 0;
            auto flush = [&]() {
                const int bt = (warp >> 2) * 32 + lane;  // 0 .. 95
                for (int x = bt; x < kStgTiles * kPostRows * 12; x += 96) {
                    const int c = x / (kStgTiles * kPostRows), rem = x % (kStgTiles * kPostRows);
                    const int tl = rem / kPostRows, row = rem % kPostRows;
                    const int srl = row / (TE * NK), se = (row / NK) % TE, sk = row % NK;
                    if (pend_E0 + se >= d.ne) continue;
                    const size_t idx = (((size_t)sk * d.ne + pend_E0 + se) * d.na + a) * kCh +
                                       (kRpt * (kPT - kStgTiles + tl) + srl) * 12 + c;
                    if (!SSE_BC(idx, (long long)d.nkz * d.ne * d.na * kCh, prm.status)) continue;
                    const float *sp = stg + ((size_t)tl * kPostRows + row) * kStgStride + 2 * c;
                    const float2 v = make_float2(sp[0], sp[1]);
                    if (pend_first) S[idx] = final_of<CT>(v);
                    else slot_add(S + idx, v);
                }
                pend = false;
            };
            auto bwait = [&](uint64_t *bar, uint32_t parity) {
                if (!bad && !mbar_wait_bounded(bar, parity, kWaitNs)) {
                    bad = true;
                    atomicOr(prm.status, kStatusTimeout);
                }
            };
            for (int g = 0; g < total; ++g, advance(cur), o = (o + 1 == slot_len) ? 0 : o + 1) {
                const int t = cur.t, vs = cur.vs, st = cur.st;
                const int gg = g_base + g, sb = gg % nbst, use = gg / nbst;
                const int E0 = t * TE;
                const bool job_first = st == 0, job_last = st == prm.nst - 1;
                if (job_first && vs > 0 && (!ENC || xw)) {
                    // the job's epilogue adds to Sigma: bring those lines to L2 while the job runs
                    constexpr int kLines = (kCh * (int)sizeof(CT) + 127) / 128;
                    constexpr int kPrefetchers = ENC ? kTcBuilders - kTcEncoders : kTcBuilders;
                    const int ptid = ENC ? (warp >> 2) * 96 + q4 * 32 + lane : tid;
                    for (int x = ptid; x < NK * TE * kLines; x += kPrefetchers) {
                        const int pt = x / kLines, ln = x % kLines, k = pt / TE, E = E0 + pt % TE;
                        if (E < d.ne && SSE_BC((((size_t)k * d.ne + E) * d.na + a) * kCh, (long long)d.nkz * d.ne * d.na * kCh, prm.status))
                            prefetch_l2((const uint8_t *)(S + (((size_t)k * d.ne + E) * d.na + a) * kCh) + ln * 128);
                    }
                }
                if (stg && !xw && pend) flush();  // the previous job's staged tiles

                // ---- X of this stage -> B buffer sb.  Warp (lane quarter q4 < 3, column block cb)
                // loads rows (i = 0, 1) and (i = 2, zero) of the four r of its quarter, columns
                // (k', t) for t in [4 cb, 4 cb + 4): thread l then holds the whole K row (i, k')
                // of B channel n = (r, t), plane re/im, with (re/im, r % 4) = l / 4 and t % 4 =
                // l % 4.  At the first stage of a pair both stages are read, the second kept. ----
                const bool pair_first = (o & 1) == 0;
                if (pair_first && xw) {
                    bwait(bar_pre, pair_ctr & 1);
                    tc_fence_after();
                }
                if (pair_first) ++pair_ctr;
                uint32_t xa[2 * NK], xb[2 * NK];  // rows (i0 | i1) and (i2 | zero), repetition k = k'
                if (xw) {
                    if (pair_first) {
                        const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + kTcPre + 4 * NK * cb;
                        tmem_ld16x128_reps<NK>(ta, xa);
                        tmem_ld16x128_reps<NK>(ta + (16u << 16), xb);
                        uint32_t na[2 * NK], nb[2 * NK];
                        tmem_ld16x128_reps<NK>(ta + 64, na);
                        tmem_ld16x128_reps<NK>(ta + 64 + (16u << 16), nb);
                        tmem_ld_wait();
                        tmem_pin(xa);
                        tmem_pin(xb);
                        tmem_pin(na);
                        tmem_pin(nb);
                        tc_fence_before();
                        mbar_arrive(bar_xfree);  // the pre-product of the next pair may overwrite X
#pragma unroll
                        for (int k = 0; k < NK; ++k) {
                            xnext[k] = na[2 * k];
                            xnext[NK + k] = na[2 * k + 1];
                            xnext[2 * NK + k] = nb[2 * k];
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < NK; ++k) {
                            xa[2 * k] = xnext[k];
                            xa[2 * k + 1] = xnext[NK + k];
                            xb[2 * k] = xnext[2 * NK + k];
                        }
                    }
                }
                // ---- the B buffer must be free: the main MMAs of its previous stage complete ----
                if (xw && use > 0) bwait(&bar_mma[sb], (use - 1) & 1);
                if (xw) {
                    // K row kk = i * Nkz + k' (3 Nkz used, the rest of the 16 zero), split into bf16 hi / lo
                    float v[16];
#pragma unroll
                    for (int k = 0; k < NK; ++k) {
                        v[k] = __uint_as_float(xa[2 * k]);
                        v[NK + k] = __uint_as_float(xa[2 * k + 1]);
                        v[2 * NK + k] = __uint_as_float(xb[2 * k]);
                    }
#pragma unroll
                    for (int k = 3 * NK; k < 16; ++k) v[k] = 0.f;
                    uint32_t hv[8], lv[8];
#pragma unroll
                    for (int x = 0; x < 8; ++x) {
                        const uint2 hl = split2_bf16(v[2 * x], v[2 * x + 1]);
                        hv[x] = hl.x;
                        lv[x] = hl.y;
                    }
                    const int pr = lane >> 4, n = (4 * q4 + ((lane >> 2) & 3)) * 12 + 4 * cb + (lane & 3);
                    if constexpr (SPLITK) {
                        // plane pr of K = 32: (hi | lo | hi) of the row, four 16-byte core-matrix rows
                        uint32_t wv[16];
                        splitk_row<3 * NK>(v, false, wv);
                        uint8_t *ph = sB + sb * (4 * GG::DA_B_PLANE) + (2 * pr) * GG::DA_B_PLANE + (n >> 3) * (2 * GG::DA_SBO_B) +
                                      (n & 7) * 16;
#pragma unroll
                        for (int kg = 0; kg < 4; ++kg)
                            *(uint4 *)(ph + kg * 128) = make_uint4(wv[4 * kg], wv[4 * kg + 1], wv[4 * kg + 2], wv[4 * kg + 3]);
                    } else {
                        uint8_t *ph = sB + sb * (4 * GG::DA_B_PLANE) + (2 * pr) * GG::DA_B_PLANE + (n >> 3) * GG::DA_SBO_B +
                                      (n & 7) * 16;
                        *(uint4 *)ph = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *(uint4 *)(ph + 128) = make_uint4(hv[4], hv[5], hv[6], hv[7]);
                        *(uint4 *)(ph + GG::DA_B_PLANE) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                        *(uint4 *)(ph + GG::DA_B_PLANE + 128) = make_uint4(lv[4], lv[5], lv[6], lv[7]);
                    }
                }
                if (xw) {
                    fence_proxy_async_smem();
                    mbar_arrive(&bar_bready[sb]);
                }

                if (job_last) {
                    // ---- epilogue of the job: Sigma += sum_j V_j dH_j^dagger (V = acc_re + i acc_im) ----
                    // the X warps see the job's MMAs done; the others (no stage work) wait at the
                    // barrier until then
                    if (xw) bwait(bar_job, job_ctr & 1);
                    ++job_ctr;
                    builders_sync<ENC>();  // every builder is done with B before the A tile overlays it
                    tc_fence_after();
                    const bool first_slot = vs == 0;
                    // A-tile role: warp -> (lane quarter, row r' of the tile); lane -> accumulator row
                    const int aq = warp & 3, arl = warp >> 2;
                    const int am = aq * 32 + lane;
                    const int ak = am / (3 * TE), aj = (am / TE) % 3, ae = am % TE;
                    // drain role: warp -> (lane quarter = tile rows, 8 of the 24 columns = 4 values s)
                    const int dq = warp & 3, dsub = warp >> 2;
                    const int drow = dq * 32 + lane;  // tile row (r', e, k)
                    const int drl = drow / (TE * NK), de = (drow / NK) % TE, dk = drow % NK;
                    const bool dlive = drow < kPostRows && E0 + de < d.ne;
                    CT *dst = S;
                    // Tile q: its A is built once the MMAs of tile q - 1 are done (one A buffer);
                    // the accumulator columns it needs are loaded before that wait, and tile
                    // q - 1's result is drained and added to Sigma after tile q is handed to the MMAs.
                    for (int q = 0; q <= kPT; ++q) {
                        const int tq = tile_ctr + q;  // CTA-wide index of tile q
                        uint32_t vr[12], vi[12];
                        uint32_t xr[4], xi[4];  // kRpt = 4: row r' = 3, columns t in [4 arl, 4 arl + 4)
                        if (q < kPT) {
                            const uint32_t ta = tmem + ((uint32_t)(aq * 32) << 16) + (uint32_t)((kRpt * q + arl) * 12);
                            tmem_ld8(ta, *reinterpret_cast<uint32_t(*)[8]>(vr));
                            tmem_ld4(ta + 8, *reinterpret_cast<uint32_t(*)[4]>(vr + 8));
                            tmem_ld8(ta + kTcAccIm, *reinterpret_cast<uint32_t(*)[8]>(vi));
                            tmem_ld4(ta + kTcAccIm + 8, *reinterpret_cast<uint32_t(*)[4]>(vi + 8));
                            if constexpr (kRpt == 4) {
                                const uint32_t tb = tmem + ((uint32_t)(aq * 32) << 16) + (uint32_t)((kRpt * q + 3) * 12 + 4 * arl);
                                tmem_ld4(tb, xr);
                                tmem_ld4(tb + kTcAccIm, xi);
                            }
                        }
                        if (q > 0) {
                            // MMAs of tile q - 1 done: its result can be drained, the A tile reused
                            bwait(&bar_post[(tq - 1) & 1], ((tq - 1) >> 1) & 1);
                            tc_fence_after();
                        }
                        tmem_ld_wait();
                        if (q < kPT) {
                            tmem_pin(vr);
                            tmem_pin(vi);
                            if constexpr (kRpt == 4) {
                                tmem_pin(xr);
                                tmem_pin(xi);
                            }
                        }
                        if (q < kPT && am < kVRows) {
                            // ---- A tile q: rows (r', e, k), K = (j, t, re/im), bf16 hi / lo ----
                            const int row = arl * (TE * NK) + ae * NK + ak;
                            uint8_t *rbase = sApost + (row >> 3) * kPostSbo + (row & 7) * 16;
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) {
                                uint32_t hw[4], lw[4];
#pragma unroll
                                for (int x = 0; x < 4; ++x) {
                                    const int t = 4 * cc + x;
                                    const uint2 hl = split2_bf16(__uint_as_float(vr[t]), __uint_as_float(vi[t]));
                                    hw[x] = hl.x;
                                    lw[x] = hl.y;
                                }
                                uint8_t *p2 = rbase + (aj * 3 + cc) * 128;
                                *(uint4 *)p2 = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                                *(uint4 *)(p2 + kPostAPlane) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                            }
                            if (aj == 2) {  // K 72..79: zero
                                *(uint4 *)(rbase + 9 * 128) = make_uint4(0u, 0u, 0u, 0u);
                                *(uint4 *)(rbase + 9 * 128 + kPostAPlane) = make_uint4(0u, 0u, 0u, 0u);
                            }
                            if constexpr (kRpt == 4) {
                                // row r' = 3 of the tile: this thread's K chunk (j, t in [4 arl, 4 arl + 4))
                                const int row3 = 3 * (TE * NK) + ae * NK + ak;
                                uint8_t *rb3 = sApost + (row3 >> 3) * kPostSbo + (row3 & 7) * 16;
                                uint32_t hw[4], lw[4];
#pragma unroll
                                for (int x = 0; x < 4; ++x) {
                                    const uint2 hl = split2_bf16(__uint_as_float(xr[x]), __uint_as_float(xi[x]));
                                    hw[x] = hl.x;
                                    lw[x] = hl.y;
                                }
                                uint8_t *p3 = rb3 + (aj * 3 + arl) * 128;
                                *(uint4 *)p3 = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                                *(uint4 *)(p3 + kPostAPlane) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                                if (aj == 2 && arl == 0) {
                                    *(uint4 *)(rb3 + 9 * 128) = make_uint4(0u, 0u, 0u, 0u);
                                    *(uint4 *)(rb3 + 9 * 128 + kPostAPlane) = make_uint4(0u, 0u, 0u, 0u);
                                }
                            }
                        }
                        tc_fence_before();
                        if (q < kPT) {
                            fence_proxy_async_smem();
                            mbar_arrive(bar_apost);
                        }
                        float pv[8];
                        if (q > 0) {
                            // ---- result of tile q - 1: rows (r', e, k) x (s, re/im); its TMEM
                            // columns are next written by tile q + 1, handed over after this ----
                            tmem_ld8(tmem + ((uint32_t)(dq * 32) << 16) + (((tq - 1) & 1) ? kTcPost1 : kTcPost0) +
                                         (uint32_t)(8 * dsub), pv);
                            tmem_ld_wait();
                            tmem_pin(pv);
                            tc_fence_before();
                        }
                        if (q > 0 && stg && q - 1 >= kPT - kStgTiles) {
                            // staged: added to Sigma during the next job (see flush)
                            if (drow < kPostRows) {
                                float *sp = stg + ((size_t)(q - 1 - (kPT - kStgTiles)) * kPostRows + drow) * kStgStride + 8 * dsub;
                                *(float4 *)sp = make_float4(pv[0], pv[1], pv[2], pv[3]);
                                *(float4 *)(sp + 4) = make_float4(pv[4], pv[5], pv[6], pv[7]);
                            }
                        } else if (q > 0 && dlive && SSE_BC((dst - S) + 3, (long long)d.nkz * d.ne * d.na * kCh, prm.status)) {
                            // the slot's FP32 contribution into Sigma: the first slot stores it, every
                            // later slot adds it with a fire-and-forget reduction at L2 (FP64 adds for
                            // complex128, the running sum then being FP64; FP32 adds for complex64)
#pragma unroll
                            for (int s2 = 0; s2 < 4; ++s2) {
                                const float2 v = make_float2(pv[2 * s2], pv[2 * s2 + 1]);
                                if (first_slot) dst[s2] = final_of<CT>(v);
                                else slot_add(dst + s2, v);
                            }
                        }
                        if (q < kPT)
                            dst = S + (((size_t)dk * d.ne + (dlive ? E0 + de : 0)) * d.na + a) * kCh + (kRpt * q + drl) * 12 +
                                  4 * dsub;
                    }
                    tile_ctr += kPT;
                    if (stg) {
                        builders_sync<ENC>();  // the staged tiles are complete
                        pend = true;
                        pend_E0 = E0;
                        pend_first = first_slot;
                    }
                }
            }
            if (stg && !xw && pend) flush();  // the unit's last job
            if (bad) s_abort[0] = 1;  // read by every thread after the unit's closing barrier
        }
        g_base += total;
        __syncthreads();
        if (s_abort[0] || s_abort[1] || *s_abort_ctl || *s_abort_prd || *s_abort_enc) {
            abort = true;
            break;
        }
    }  // units

    // ---- teardown: nothing of ours may still be in flight when the CTA exits ----
    if (abort && ctl && lane == 0) {
        mma_commit(bar_fin);  // arrives once every MMA issued so far is done
        mbar_wait_bounded(bar_fin, 0, kWaitNs);
    }
    if (abort && prd && lane == 0) {
        for (int b = 0; b < kTcRing; ++b)
            if (last_g[b] >= 0) mbar_wait_bounded(&bar_g[b], (last_g[b] / kTcRing) & 1, kWaitNs);
        if (slot_cp > 0) {
            mbar_wait_bounded(bar_slot, (slot_cp - 1) & 1, kWaitNs);
            mbar_wait_bounded(bar_tab, (slot_cp - 1) & 1, kWaitNs);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Shared memory of the warp-specialised kernel: the B stages (the epilogue's post-product
// A tile overlays them), the G-slice ring, in the encoding form the raw G ring, the
// pre-product's dH operand, the direct table, the post-product's conj(dH) operand and the
// barriers.
template <int NK, bool ENC>
uint32_t tc_layout(const Dims &d, size_t cbytes, MixParams &prm, uint32_t bregion, uint32_t stg_bytes) {
    using GG = Geo<NK>;
    uint32_t off = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        off = (off + align - 1) / align * align;
        const uint32_t at = off;
        off += bytes;
        return at;
    };
    prm.off_b = take(bregion, 1024);
    prm.off_g = take(kTcRing * kTcPairBytes, 1024);
    prm.off_x = ENC ? take((uint32_t)(kTcRing * 2 * NK * kCh * cbytes), 128) : 0;
    prm.off_a = take(2 * 8192, 1024);
    const uint32_t rows = (uint32_t)(d.nw + 2 * GG::DA_TE - 2);
    prm.off_df = take(2u * 2u * GG::DA_GROUPS * 2u * rows * 16u, 1024);
    prm.off_dh = 0;
    prm.off_bp = take(2 * kPostBPlane, 1024);
    prm.off_bar = take(kTcBarBytes + 8 + 2 * kMaxSlots * 4, 8);
    prm.off_stg = stg_bytes ? take(stg_bytes, 128) : 0u;
    prm.g_stage = 0;
    return off;
}
template <int NK, bool ENC>
uint32_t tc_smem_bytes(const Dims &d, size_t cbytes, MixParams &prm) {
    using GG = Geo<NK>;
    // B buffers (the post-product A tile overlays them): a third one in the encoding form
    // when the whole layout still fits
    const uint32_t nv = 2 * kPostAPlane;
    const uint32_t b2 = kTcBStages * 4 * GG::DA_B_PLANE, b3 = kTcBStagesMax * 4 * GG::DA_B_PLANE;
    if (ENC) {
        const uint32_t s3 = tc_layout<NK, ENC>(d, cbytes, prm, b3 > nv ? b3 : nv, 0u);
        if (s3 <= 232448u) {
            prm.nbst = kTcBStagesMax;
            return s3;
        }
    }
    prm.nbst = kTcBStages;
    if (!ENC) {
        // the staging of the last post-product tiles, where it fits
        const uint32_t sb = (uint32_t)(kStgTiles * 3 * GG::DA_TE * NK * kStgStride * 4);
        const uint32_t ss = tc_layout<NK, ENC>(d, cbytes, prm, b2 > nv ? b2 : nv, sb);
        if (ss <= 232448u) return ss;
    }
    return tc_layout<NK, ENC>(d, cbytes, prm, b2 > nv ? b2 : nv, 0u);
}

template <int NK>
uint32_t mixed_smem_bytes(const Dims &d, size_t cbytes, MixParams &prm) {
    using GG = Geo<NK>;
    uint32_t off = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        off = (off + align - 1) / align * align;
        const uint32_t at = off;
        off += bytes;
        return at;
    };
    const uint32_t need_v = 2 * kRowsMax * kVStride * 4;
    const uint32_t dtmp = (uint32_t)(NK * d.nw * 9 * 8);
    prm.g_stage = (uint32_t)(GG::P * NK * kCh * cbytes);
    if (GG::DA) {
        // B stages, raw G, the direct table (the drained accumulators overlay it)
        const uint32_t bsz = 2 * 4 * GG::DA_B_PLANE;
        prm.off_b = take(bsz, 1024);
        prm.off_a = prm.off_b;
        prm.off_g = take(2 * prm.g_stage, 128);
        prm.off_x = 0;
        const uint32_t rows = (uint32_t)(d.nw + 2 * GG::DA_TE - 2);
        const uint32_t tab = 2u * 2u * GG::DA_GROUPS * 2u * rows * 16u;
        prm.off_df = take(tab > need_v ? tab : need_v, 1024);
        prm.off_dh = take(3 * kCh * 8, 16);
        prm.off_bar = take(128 + 8 + 2 * kMaxSlots * 4, 8);
        if (dtmp > bsz) return 0xFFFFFFFFu;
        return off;
    }
    // B and A stage buffers are contiguous; the drained accumulators and the unrotated
    // Dt table of a job overlay them (never while MMAs read them)
    const uint32_t ab = 2 * 2 * GG::B_PLANE + 2 * 4 * GG::A_PLANE;
    prm.off_b = take(ab > need_v ? ab : need_v, 1024);
    prm.off_a = prm.off_b + 2 * 2 * GG::B_PLANE;
    prm.off_g = take(2 * prm.g_stage, 128);
    const uint32_t grp = ((uint32_t)(d.nw + GG::P - 1) * (GG::KST * 4 + 16) + 127u) / 128u * 128u + 16u;
    const uint32_t tab = (uint32_t)(3 * NK) * grp;
    prm.off_df = take(tab, 16);
    prm.off_dh = take(3 * kCh * 8, 16);
    prm.off_bar = take(128 + 8 + 2 * kMaxSlots * 4, 8);
    prm.off_x = 0;
    if (dtmp > (ab > need_v ? ab : need_v)) return 0xFFFFFFFFu;
    return off;
}

// One instance descriptor from a plan and its buffers; the requested signs are packed
// into slots 0 and 1.  Returns false when no sign is requested.
template <int NK, bool V3>
bool fill_inst(InstDesc &I, const Plan &p, const sse_io &io, int tpc, bool dfull) {
    using GG = Geo<NK>;
    constexpr int TE = V3 ? GG::DA_TE : GG::TE;
    const bool do_gt = io.S_gt != nullptr, do_lt = io.S_lt != nullptr;
    I.nsign = (int)do_gt + (int)do_lt;
    if (I.nsign == 0) return false;
    I.G[0] = do_gt ? io.G_gt : io.G_lt;
    I.D[0] = do_gt ? io.D_gt : io.D_lt;
    I.S[0] = do_gt ? io.S_gt : io.S_lt;
    I.G[1] = io.G_lt;
    I.D[1] = io.D_lt;
    I.S[1] = io.S_lt;
    I.dH = p.geo.dH;
    I.neigh = p.geo.neigh;
    I.rev = dfull ? p.d_rev : nullptr;
    I.na = p.d.na;
    I.ne = p.d.ne;
    I.nb = p.d.nb;
    I.nqz = p.d.nqz;
    I.ntiles = (I.ne + TE - 1) / TE;
    I.tiles_per_cta = tpc < 1 ? 1 : (tpc > I.ntiles ? I.ntiles : tpc);
    // the workspace: stored G slices (Nkz = 5 only), then the slot tables
    const size_t sign_bytes = NK == 5 ? ((size_t)p.d.ne * p.d.na + 1) * 8192 : 0;
    const size_t tab_sign = (size_t)p.d.na * p.d.nb * tc_entry_bytes(p.d.nw);
    const uint8_t *ws = (const uint8_t *)p.mixed_ws;
    I.gws[0] = (ws && NK == 5) ? ws + (do_gt ? 0 : sign_bytes) : nullptr;
    I.gws[1] = (ws && NK == 5) ? ws + sign_bytes : nullptr;
    I.sws[0] = ws ? ws + 2 * sign_bytes + (do_gt ? 0 : tab_sign) : nullptr;
    I.sws[1] = ws ? ws + 2 * sign_bytes + tab_sign : nullptr;
    I.nchunks = (I.ntiles + I.tiles_per_cta - 1) / I.tiles_per_cta;
    return true;
}

long long inst_units(const InstDesc &I) { return (long long)I.nsign * I.na * I.nchunks; }

// The warp-specialised kernel instance for a B-buffer count (three only in the encoding
// form), and its launch with the count tc_smem_bytes chose.
template <int NK, typename CT, bool ENC, int BST>
auto tc_kernel_of() {
    if constexpr (BST == kTcBStagesMax && !ENC) return sse_tc_kernel<NK, CT, ENC, kTcBStages>;
    else return sse_tc_kernel<NK, CT, ENC, BST>;
}
template <int NK, typename CT>
void launch_tc(const MixParams &prm, unsigned grid, uint32_t smem, cudaStream_t st) {
    constexpr bool ENC = NK < 5;
    if (ENC && prm.nbst == kTcBStagesMax)
        tc_kernel_of<NK, CT, ENC, kTcBStagesMax>()<<<grid, kTcThreads, smem, st>>>(prm);
    else
        tc_kernel_of<NK, CT, ENC, kTcBStages>()<<<grid, kTcThreads, smem, st>>>(prm);
}

template <int NK, typename CT, bool V3>
sse_status prepare(MixParams &prm, uint32_t &smem, const Dims &d, int32_t *status) {
    using GG = Geo<NK>;
    constexpr bool ENC = V3 && NK < 5;  // below Nkz = 5 the warp-specialised form encodes G itself
    smem = V3 ? tc_smem_bytes<NK, ENC>(d, sizeof(CT), prm) : mixed_smem_bytes<NK>(d, sizeof(CT), prm);
    if (smem > 232448u) {
        set_error("mixed mode: Nkz=%d, Nw=%d needs more shared memory than one SM has", d.nkz, d.nw);
        return SSE_E_INVALID_ARG;
    }
    prm.status = status;
    prm.nkz = d.nkz;
    prm.nw = d.nw;
    prm.omega_first = d.omega_first;
    prm.nst = V3 ? GG::DA_TE + d.nw - 1 : (GG::TE + d.nw - 1 + GG::P - 1) / GG::P;
    cudaError_t e;
    if constexpr (V3)
        e = prm.nbst == kTcBStagesMax
                ? cudaFuncSetAttribute(tc_kernel_of<NK, CT, ENC, kTcBStagesMax>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                : cudaFuncSetAttribute(tc_kernel_of<NK, CT, ENC, kTcBStages>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        e = cudaFuncSetAttribute(sse_mixed_kernel<NK, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mixed kernel)");
    return SSE_OK;
}

// Fill the plan's workspace for every requested sign of one instance: G re-encoded for the
// pre-product and the slot tables.
template <int NK, typename CT>
sse_status split_g(const Plan &p, const sse_io &io, cudaStream_t st, bool dfull) {
    const size_t sign_bytes = NK == 5 ? ((size_t)p.d.ne * p.d.na + 1) * 8192 : 0;
    const size_t tab_sign = (size_t)p.d.na * p.d.nb * tc_entry_bytes(p.d.nw);
    const void *gs[2] = {io.S_gt ? io.G_gt : nullptr, io.S_lt ? io.G_lt : nullptr};
    const void *ds[2] = {io.D_gt, io.D_lt};
    const uint32_t tsmem = 3 * kDhJ * 8 + 5 * p.d.nw * 9 * 8;
    if (p.d.nkz != NK) return set_error("mixed mode: workspace pass for the wrong Nkz"), SSE_E_INVALID_ARG;
    for (int s = 0; s < 2; ++s) {
        if (!gs[s]) continue;
        const long long slices = (long long)p.d.ne * p.d.na;
        if (slices > 0x7fffffffLL || (long long)p.d.na * p.d.nb > 0x7fffffffLL)
            return set_error("mixed mode: instance too large"), SSE_E_INVALID_ARG;
        uint8_t *ws = (uint8_t *)p.mixed_ws;
        if (NK == 5)  // below Nkz = 5 the kernel encodes G itself
            sse_split_g_kernel<CT><<<(unsigned)slices, 256, 0, st>>>((const CT *)gs[s], ws + s * sign_bytes, p.d.ne,
                                                                    p.d.na, p.d.nkz);
        sse_slot_tables_kernel<NK, CT><<<(unsigned)(p.d.na * p.d.nb), 256, tsmem, st>>>(
            (const CT *)ds[s], (const CT *)p.geo.dH, p.geo.neigh, dfull ? p.d_rev : nullptr,
            ws + 2 * sign_bytes + s * tab_sign, p.d.na, p.d.nb, p.d.nqz, p.d.nw, p.d_status);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch the workspace kernels");
    return SSE_OK;
}

bool aligned16(const sse_io &io) {
    return ((((uintptr_t)io.G_gt | (uintptr_t)io.G_lt)) & 15u) == 0;
}

template <int NK, typename CT, bool V3>
sse_status launch_nk(Plan &p, const sse_io &io, cudaStream_t st, bool dfull) {
    using GG = Geo<NK>;
    MixParams prm{};
    uint32_t smem = 0;
    sse_status rs = prepare<NK, CT, V3>(prm, smem, p.d, p.d_status);
    if (rs != SSE_OK) return rs;
    if (!aligned16(io)) return set_error("mixed mode: G buffers must be 16-byte aligned"), SSE_E_INVALID_ARG;
    // tiles per unit: enough units for several waves over the SMs; the warp-specialised form
    // also keeps the Sigma tiles of the units in flight (one per SM) within half the L2, so
    // that a unit's sum over neighbour slots reduces into lines still in L2
    int sms = 148, l2 = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, p.device);
    constexpr int TE = V3 ? GG::DA_TE : GG::TE;
    const int ntiles = (p.d.ne + TE - 1) / TE;
    const long long per_chunk = (long long)((io.S_gt != nullptr) + (io.S_lt != nullptr)) * p.d.na;
    int tpc = ntiles;
    while (tpc > 1 && per_chunk * ((ntiles + tpc - 1) / tpc) < 8LL * sms) tpc = (tpc + 1) / 2;
    if (V3 && l2 > 0) {
        const long long tile_bytes = (long long)TE * NK * kCh * sizeof(CT);
        while (tpc > 1 && (long long)sms * tpc * tile_bytes > l2 / 2) tpc = (tpc + 1) / 2;
    }
    // SSE_TILES_PER_UNIT overrides the choice (tuning experiments; values are clamped to
    // [1, tiles per atom] by fill_inst)
    if (const char *env = getenv("SSE_TILES_PER_UNIT"))
        if (atoi(env) > 0) tpc = atoi(env);
    if (!fill_inst<NK, V3>(prm.inst[0], p, io, tpc, dfull)) return SSE_OK;
    prm.n_inst = 1;
    prm.inject = take_inject(SSE_INJECT_STALL) ? 1 : 0;
    prm.inst[0].unit_begin = 0;
    prm.total_units = inst_units(prm.inst[0]);
    prm.queue = nullptr;
    if (prm.total_units > 0x7fffffffLL) return set_error("mixed mode: grid too large"), SSE_E_INVALID_ARG;
    const int ts = timing_slot(p);
    timing_mark(p, ts, 0, st);
    if (V3) {
        rs = split_g<NK, CT>(p, io, st, dfull);
        if (rs != SSE_OK) return rs;
    }
    timing_mark(p, ts, 1, st);
    if constexpr (V3)
        launch_tc<NK, CT>(prm, (unsigned)prm.total_units, smem, st);
    else
        sse_mixed_kernel<NK, CT><<<(unsigned)prm.total_units, kThreads, smem, st>>>(prm);
    timing_mark(p, ts, 2, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch sse_mixed_kernel");
    p.tile_e = TE;
    return SSE_OK;
}

// Persistent launches over many instances: one CTA per SM pulls units from a counter.
template <int NK, typename CT, bool V3>
sse_status launch_batch_nk(Plan *const *plans, const sse_io *ios, const int *order, int n, int tpc,
                           int32_t *queue, int32_t *status, cudaStream_t st) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plans[0]->device);
    for (int base = 0; base < n; base += kMaxInst) {
        MixParams prm{};
        uint32_t smem = 0;
        sse_status rs = prepare<NK, CT, V3>(prm, smem, plans[order[base]]->d, status);
        if (rs != SSE_OK) return rs;
        long long units = 0;
        int m = 0;
        for (int x = base; x < n && x < base + kMaxInst; ++x) {
            const Plan &p = *plans[order[x]];
            const sse_io &io = ios[order[x]];
            if (!aligned16(io)) return set_error("mixed mode: G buffers must be 16-byte aligned"), SSE_E_INVALID_ARG;
            if (!fill_inst<NK, V3>(prm.inst[m], p, io, tpc, false)) continue;
            if (V3) {
                rs = split_g<NK, CT>(p, io, st, false);
                if (rs != SSE_OK) return rs;
            }
            prm.inst[m].unit_begin = units;
            units += inst_units(prm.inst[m]);
            ++m;
        }
        if (m == 0) continue;
        prm.n_inst = m;
        prm.inject = (base == 0 && take_inject(SSE_INJECT_STALL)) ? 1 : 0;
        prm.total_units = units;
        prm.queue = queue;
        cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "reset the work counter");
        const long long grid = units < sms ? units : sms;
        if constexpr (V3)
            launch_tc<NK, CT>(prm, (unsigned)grid, smem, st);
        else
            sse_mixed_kernel<NK, CT><<<(unsigned)grid, kThreads, smem, st>>>(prm);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "launch persistent sse_mixed_kernel");
    }
    return SSE_OK;
}

template <typename CT>
sse_status launch_dtype(Plan &p, const sse_io &io, cudaStream_t st, bool dfull) {
    // the warp-specialised form when the plan has its workspace, else the single-role form
    const bool ws = p.mixed_ws != nullptr;
    switch (p.d.nkz) {
        case 1: return ws ? launch_nk<1, CT, true>(p, io, st, dfull) : launch_nk<1, CT, false>(p, io, st, dfull);
        case 2: return ws ? launch_nk<2, CT, true>(p, io, st, dfull) : launch_nk<2, CT, false>(p, io, st, dfull);
        case 3: return ws ? launch_nk<3, CT, true>(p, io, st, dfull) : launch_nk<3, CT, false>(p, io, st, dfull);
        case 4: return ws ? launch_nk<4, CT, true>(p, io, st, dfull) : launch_nk<4, CT, false>(p, io, st, dfull);
        case 5: return ws ? launch_nk<5, CT, true>(p, io, st, dfull) : launch_nk<5, CT, false>(p, io, st, dfull);
        default:
            set_error("mixed mode supports Nkz <= 5 (got %d)", p.d.nkz);
            return SSE_E_INVALID_ARG;
    }
}

template <int NK, typename CT>
sse_status launch_batch_form(Plan *const *plans, const sse_io *ios, const int *order, int n, int tpc,
                             int32_t *queue, int32_t *status, cudaStream_t st) {
    // the warp-specialised form needs each plan's workspace for itself: every plan once
    bool all_ws = true;
    for (int x = 0; x < n && all_ws; ++x) {
        all_ws = plans[order[x]]->mixed_ws != nullptr;
        for (int y = 0; y < x && all_ws; ++y) all_ws = plans[order[y]] != plans[order[x]];
    }
    return all_ws ? launch_batch_nk<NK, CT, true>(plans, ios, order, n, tpc, queue, status, st)
                  : launch_batch_nk<NK, CT, false>(plans, ios, order, n, tpc, queue, status, st);
}

template <typename CT>
sse_status launch_batch_dtype(Plan *const *plans, const sse_io *ios, const int *order, int n, int tpc,
                              int32_t *queue, int32_t *status, cudaStream_t st) {
    switch (plans[order[0]]->d.nkz) {
        case 1: return launch_batch_form<1, CT>(plans, ios, order, n, tpc, queue, status, st);
        case 2: return launch_batch_form<2, CT>(plans, ios, order, n, tpc, queue, status, st);
        case 3: return launch_batch_form<3, CT>(plans, ios, order, n, tpc, queue, status, st);
        case 4: return launch_batch_form<4, CT>(plans, ios, order, n, tpc, queue, status, st);
        case 5: return launch_batch_form<5, CT>(plans, ios, order, n, tpc, queue, status, st);
        default:
            set_error("mixed mode supports Nkz <= 5");
            return SSE_E_INVALID_ARG;
    }
}

// Shared memory of both forms for one Nkz: the single-role form's (the plan is valid only if
// it fits: the no-alloc entry and batches holding a plan twice use it) and the
// warp-specialised form's.
template <int NK>
void smem_of(const Dims &d, size_t cb, uint32_t &single, uint32_t &ws) {
    MixParams prm{};
    single = mixed_smem_bytes<NK>(d, cb, prm);
    ws = tc_smem_bytes<NK, (NK < 5)>(d, cb, prm);
}

}  // namespace

sse_status mixed_plan_init(Plan &p) {
    const Dims &d = p.d;
    if (d.nkz < 1 || d.nkz > 5) {
        set_error("mixed mode supports Nkz <= 5 (got %d)", d.nkz);
        return SSE_E_INVALID_ARG;
    }
    if (d.nb > kMaxSlots) {
        set_error("mixed mode supports nb_max <= %d (got %d)", kMaxSlots, d.nb);
        return SSE_E_INVALID_ARG;
    }
    uint32_t smem = 0, smem_ws = 0;
    const size_t cb = elem_bytes(p.geo.dtype);
    switch (d.nkz) {
        case 1: smem_of<1>(d, cb, smem, smem_ws); p.tile_e = Geo<1>::TE; break;
        case 2: smem_of<2>(d, cb, smem, smem_ws); p.tile_e = Geo<2>::TE; break;
        case 3: smem_of<3>(d, cb, smem, smem_ws); p.tile_e = Geo<3>::TE; break;
        case 4: smem_of<4>(d, cb, smem, smem_ws); p.tile_e = Geo<4>::TE; break;
        default: smem_of<5>(d, cb, smem, smem_ws); p.tile_e = Geo<5>::TE; break;
    }
    if (smem > 232448u) {
        set_error("mixed mode: Nkz=%d, Nw=%d needs more shared memory than one SM has", d.nkz, d.nw);
        return SSE_E_INVALID_ARG;
    }
    // the warp-specialised tensor-core form when its tiles fit (Nw <= 50 at Nkz = 5), with a
    // workspace; otherwise the single-role form above
    if (smem_ws <= 232448u) {
        // workspace, per sign: at Nkz = 5 G re-encoded for the pre-product plus a zero slice
        // (below that the kernel encodes G itself), then the slot tables of every (atom, slot)
        const size_t sign_bytes = d.nkz == 5 ? ((size_t)d.ne * d.na + 1) * 8192 : 0;
        const size_t tab_sign = (size_t)d.na * d.nb * tc_entry_bytes(d.nw);
        const size_t bytes = 2 * sign_bytes + 2 * tab_sign;
        cudaError_t e = take_inject(SSE_INJECT_ALLOC_FAIL) ? cudaErrorMemoryAllocation : cudaMalloc(&p.mixed_ws, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p.mixed_ws = nullptr;
            set_error("cudaMalloc of %zu bytes for the mixed workspace failed", bytes);
            return SSE_E_OUT_OF_MEMORY;
        }
        p.mixed_ws_bytes = bytes;
        p.workspace_bytes += (int64_t)p.mixed_ws_bytes;
        p.tile_e = Geo<5>::DA_TE;
        for (int s2 = 0; s2 < 2 && sign_bytes > 0; ++s2) {
            e = cudaMemset((uint8_t *)p.mixed_ws + s2 * sign_bytes + (size_t)d.ne * d.na * 8192, 0, 8192);
            if (e != cudaSuccess) return cuda_fail(e, "clear the zero slice");
        }
    }
    return SSE_OK;
}

void mixed_plan_free(Plan &p) {
    if (p.mixed_ws) cudaFree(p.mixed_ws);
    p.mixed_ws = nullptr;
    p.mixed_ws_bytes = 0;
}

sse_status launch_mixed(Plan &p, const sse_io &io, cudaStream_t st, bool dfull) {
    if (p.geo.dtype == SSE_C128) return launch_dtype<double2>(p, io, st, dfull);
    return launch_dtype<float2>(p, io, st, dfull);
}

sse_status launch_mixed_batch(Plan *const *plans, const sse_io *ios, const int *order, int n, int tpc,
                              int32_t *queue, int32_t *status, cudaStream_t st) {
    if (n <= 0) return SSE_OK;
    if (plans[order[0]]->geo.dtype == SSE_C128) return launch_batch_dtype<double2>(plans, ios, order, n, tpc, queue, status, st);
    return launch_batch_dtype<float2>(plans, ios, order, n, tpc, queue, status, st);
}

}  // namespace sse
