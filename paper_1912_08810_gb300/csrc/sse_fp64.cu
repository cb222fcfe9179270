// FP64 direct form of the electron scattering self-energy (Eq. 3) -- the plain GPU
// baseline and the oracle-matching reference mode.
//
// One CTA computes one output block Sigma[k, E, a] (144 complex channels, one thread
// per channel) for one sign.  For each neighbour slot b (f = neigh[a, b]):
//   1. correlation, per channel c = (r, t):
//        Y_ij[c] = sum_{q, w} Dt[q, w, a, b, i, j] * G[(k - q) mod nkz, E - w - omega_first, f][c]
//      (nine accumulators per thread; the G row of 144 channels is one coalesced load)
//   2. Z_i = sum_j Y_ij . dH_j^dagger          (nine 12x12 products through shared memory)
//   3. Sigma += sum_i dH_i . Z_i              (three 12x12 products)
// This is Eq. 3 regrouped by linearity: dH_i (sum_{q,w} Dt_ij G) dH_j^dagger.  Per
// (point, slot) it issues exactly the algorithmic count of the redundancy-removed form
// (Section 3): 9 * 144 complex MACs per valid (q, w) plus twelve 12x12 products.
// Every multiply and add is FP64 (DFMA); the FP64 pipe bounds this kernel.
#include <cuda_runtime.h>

#include "sse_internal.h"

namespace sse {
namespace {

template <typename CT>
__device__ __forceinline__ double2 ld(const CT *p);
template <>
__device__ __forceinline__ double2 ld<double2>(const double2 *p) { return __ldg(p); }
template <>
__device__ __forceinline__ double2 ld<float2>(const float2 *p) {
    float2 v = __ldg(p);
    return make_double2(v.x, v.y);
}

template <typename CT>
__device__ __forceinline__ void st(CT *p, double2 v);
template <>
__device__ __forceinline__ void st<double2>(double2 *p, double2 v) { *p = v; }
template <>
__device__ __forceinline__ void st<float2>(float2 *p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

// acc += a * b
__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += a * conj(b)
__device__ __forceinline__ void cmac_conj(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
}

constexpr int kThreads = 160;  // 144 channels rounded up to whole warps

template <typename CT>
__global__ void __launch_bounds__(kThreads)
sse_fp64_direct_kernel(const int32_t *__restrict__ neigh, const CT *__restrict__ dH,
                       const CT *__restrict__ G0, const CT *__restrict__ D0, CT *__restrict__ S0,
                       const CT *__restrict__ G1, const CT *__restrict__ D1, CT *__restrict__ S1,
                       Dims d, int32_t *status) {
    __shared__ double2 s_dh[kN3D][kBlk];
    __shared__ double2 s_y[kN3D * kN3D][kBlk];
    __shared__ double2 s_z[kN3D][kBlk];

    const CT *G = blockIdx.y == 0 ? G0 : G1;
    const CT *D = blockIdx.y == 0 ? D0 : D1;
    CT *S = blockIdx.y == 0 ? S0 : S1;

    // point index with the atom fastest, so neighbouring CTAs share G rows in L2
    const int64_t p = blockIdx.x;
    const int a = (int)(p % d.na);
    const int e = (int)((p / d.na) % d.ne);
    const int k = (int)(p / ((int64_t)d.na * d.ne));

    const int c = threadIdx.x;
    const bool active = c < kBlk;
    const int r = c / kNorb, s = c % kNorb;
    double2 acc = make_double2(0.0, 0.0);

    for (int slot = 0; slot < d.nb; ++slot) {
        const int f = __ldg(neigh + (size_t)a * d.nb + slot);
        if (f < 0) continue;  // empty slot (uniform over the CTA)
        if (!SSE_BC(f, d.na, status)) continue;
        const CT *dh = dH + ((size_t)a * d.nb + slot) * kN3D * kBlk;
        for (int x = threadIdx.x; x < kN3D * kBlk; x += kThreads) s_dh[x / kBlk][x % kBlk] = ld(dh + x);

        double2 y[kN3D * kN3D];
#pragma unroll
        for (int ij = 0; ij < kN3D * kN3D; ++ij) y[ij] = make_double2(0.0, 0.0);
        if (active) {
            for (int q = 0; q < d.nqz; ++q) {
                int kk = (k - q) % d.nkz;
                if (kk < 0) kk += d.nkz;
                const CT *gq = G + ((size_t)kk * d.ne) * d.na * kBlk + (size_t)f * kBlk + c;
                const CT *dq = D + (((size_t)q * d.nw) * d.na + a) * d.nb * 9 + (size_t)slot * 9;
                // frequencies whose E' = E - w - omega_first lies on the grid: w_lo drops E' above
                // it (negative omega_first), w_hi those below it
                const int w_lo = max(0, e - d.omega_first - (d.ne - 1));
                const int w_hi = min(d.nw - 1, e - d.omega_first);
                for (int w = w_lo; w <= w_hi; ++w) {
                    const int ep = e - w - d.omega_first;
                    const CT *gp = gq + (size_t)ep * d.na * kBlk;
                    const CT *dw = dq + (size_t)w * d.na * d.nb * 9;
                    if (!SSE_BC(gp - G, (long long)d.nkz * d.ne * d.na * kBlk, status) ||
                        !SSE_BC(dw + 8 - D, (long long)d.nqz * d.nw * d.na * d.nb * 9, status))
                        continue;
                    const double2 g = ld(gp);
#pragma unroll
                    for (int ij = 0; ij < 9; ++ij) cmac(y[ij], ld(dw + ij), g);
                }
            }
#pragma unroll
            for (int ij = 0; ij < 9; ++ij) s_y[ij][c] = y[ij];
        }
        __syncthreads();
        if (active) {
            // Z_i[r, s] = sum_j sum_t Y_ij[r, t] conj(dH_j[s, t])
#pragma unroll
            for (int i = 0; i < kN3D; ++i) {
                double2 z = make_double2(0.0, 0.0);
#pragma unroll
                for (int j = 0; j < kN3D; ++j)
#pragma unroll
                    for (int t = 0; t < kNorb; ++t) cmac_conj(z, s_y[i * 3 + j][r * kNorb + t], s_dh[j][s * kNorb + t]);
                s_z[i][c] = z;
            }
        }
        __syncthreads();
        if (active) {
            // Sigma[r, s] += sum_i sum_u dH_i[r, u] Z_i[u, s]
#pragma unroll
            for (int i = 0; i < kN3D; ++i)
#pragma unroll
                for (int u = 0; u < kNorb; ++u) cmac(acc, s_dh[i][r * kNorb + u], s_z[i][u * kNorb + s]);
        }
        __syncthreads();
    }
    if (active && SSE_BC((size_t)p * kBlk + c, (long long)d.nkz * d.ne * d.na * kBlk, status))
        st(S + (size_t)p * kBlk + c, acc);
}

}  // namespace

sse_status launch_fp64_direct(const Plan &p, const sse_io &io, cudaStream_t st) {
    const Dims &d = p.d;
    const int64_t points = (int64_t)d.nkz * d.ne * d.na;
    if (points == 0) return SSE_OK;
    if (points > 0x7fffffffLL) {
        set_error("FP64 direct kernel: %lld points exceed the grid limit", (long long)points);
        return SSE_E_INVALID_ARG;
    }
    // sign 0 = '>' and sign 1 = '<'; a skipped sign is folded away by launching one row
    const bool do_gt = io.S_gt != nullptr, do_lt = io.S_lt != nullptr;
    const int nsign = (int)do_gt + (int)do_lt;
    if (nsign == 0) return SSE_OK;
    dim3 grid((unsigned)points, nsign);
    if (p.geo.dtype == SSE_C128) {
        const double2 *g0 = (const double2 *)(do_gt ? io.G_gt : io.G_lt), *d0 = (const double2 *)(do_gt ? io.D_gt : io.D_lt);
        double2 *s0 = (double2 *)(do_gt ? io.S_gt : io.S_lt);
        sse_fp64_direct_kernel<double2><<<grid, kThreads, 0, st>>>(
            p.geo.neigh, (const double2 *)p.geo.dH, g0, d0, s0, (const double2 *)io.G_lt,
            (const double2 *)io.D_lt, (double2 *)io.S_lt, d, p.d_status);
    } else {
        const float2 *g0 = (const float2 *)(do_gt ? io.G_gt : io.G_lt), *d0 = (const float2 *)(do_gt ? io.D_gt : io.D_lt);
        float2 *s0 = (float2 *)(do_gt ? io.S_gt : io.S_lt);
        sse_fp64_direct_kernel<float2><<<grid, kThreads, 0, st>>>(
            p.geo.neigh, (const float2 *)p.geo.dH, g0, d0, s0, (const float2 *)io.G_lt,
            (const float2 *)io.D_lt, (float2 *)io.S_lt, d, p.d_status);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch sse_fp64_direct_kernel");
    return SSE_OK;
}

}  // namespace sse
