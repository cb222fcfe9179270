// The phonon scattering self-energy Pi^{<>} (Eq. 5 for the off-diagonal blocks, Eq. 4 for
// the diagonal ones, Section 2), FP64 throughout:
//   Pi[q, w, a, slot, i, j] = sum_k sum_{E : E' = E + (w + omega_first) < ne}
//        tr{ dH[a,slot,i]^dagger . Ga[(k + q) mod nkz, E', a] . dH[a,slot,j] . Gb[k, E, b] }
//   Pi[q, w, a, nb, i, j]   = - sum_{slots with b >= 0} Pi[q, w, a, slot, i, j]
// with b = neigh[a, slot], (Ga, Gb) = (G^>, G^<) for Pi^> and (G^<, G^>) for Pi^<.
//
// The trace is a dot product over the 144 channels c = (r, s):
//   tr{V_i U_j} = sum_c V_i[r, s] U_j[s, r],  V_i = dH_i^dagger Ga,  U_j = dH_j Gb,
// so per bond Pi is a correlation over (k, E) of 144-channel vectors with output (q, w).
// One CTA per (atom, sign) walks the atom's neighbour slots.  For each (q, k) it streams the
// energies once: at step E it forms U_j^T[k, E] and the newest V_i row, V_i[k + q, E + omega_max],
// keeps the last Nw rows of V_i in a shared-memory ring, and thread (w, channel subset)
// accumulates the nine (i, j) dot products of V_i[E + omega_w] with U_j^T[E] over its
// channels.  Channels go in chunks of 48 (four rows r of the block) so the ring stays
// within shared memory.  Each V_i and U_j block is formed Nqz times (once per (q, k) that
// needs it): about 25 % more work than the correlation alone at Nqz = 5, Nw = 32, and no
// workspace.  FP64 pipe bound (the GB300 FP64 rate is far below its FP32 rate).
#include <cuda_runtime.h>

#include "sse_internal.h"

namespace sse {
namespace {

constexpr int kPiThreads = 256;
constexpr int kChunk = 48;  // channels per pass: rows r in [4m, 4m + 4), all s

template <typename CT>
__device__ __forceinline__ double2 ldd(const CT *p);
template <>
__device__ __forceinline__ double2 ldd<double2>(const double2 *p) { return __ldg(p); }
template <>
__device__ __forceinline__ double2 ldd<float2>(const float2 *p) {
    const float2 v = __ldg(p);
    return make_double2(v.x, v.y);
}
template <typename CT>
__device__ __forceinline__ void std_(CT *p, double2 v);
template <>
__device__ __forceinline__ void std_<double2>(double2 *p, double2 v) { *p = v; }
template <>
__device__ __forceinline__ void std_<float2>(float2 *p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {  // acc += a b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac_cj(double2 &acc, double2 a, double2 b) {  // acc += conj(a) b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

struct PiArgs {
    const void *Ga[2], *Gb[2];  // per sign slot (0: first requested sign)
    void *Pi[2];
    const int32_t *neigh;
    const void *dH;
    int32_t nkz, nqz, ne, nw, na, nb, omega_first;
    int32_t cs;  // channel subsets per w (threads = nw * cs <= 256, kChunk % cs == 0)
    int32_t *status;  // bounds-checked build: index violations
};

template <typename CT>
__global__ void __launch_bounds__(kPiThreads, 2) sse_pi_kernel(const __grid_constant__ PiArgs p) {
    extern __shared__ __align__(16) uint8_t smem[];
    double2 *s_dh = (double2 *)smem;                // [3][144] dH_i of the slot
    double2 *s_ga = s_dh + 3 * 144;                 // [144] Ga block of the newest V row
    double2 *s_gb = s_ga + 144;                     // [144] Gb block of this step
    double2 *s_u = s_gb + 144;                      // [3][kChunk] U_j^T of this step
    double2 *s_red = s_u + 3 * kChunk;              // [nw * cs][9] for the reduction over subsets
    double2 *s_ring = s_red + (size_t)p.nw * p.cs * 9;  // [nw][3][kChunk] ring of V_i rows

    const int a = blockIdx.x, sg = blockIdx.y, tid = threadIdx.x;
    const CT *Ga = (const CT *)p.Ga[sg];
    const CT *Gb = (const CT *)p.Gb[sg];
    CT *Pi = (CT *)p.Pi[sg];
    const CT *dH = (const CT *)p.dH;
    const int nw = p.nw, cs = p.cs, nb1 = p.nb + 1;
    const int omega_max = p.omega_first + nw - 1;
    const bool worker = tid < nw * cs;
    const int w = tid / cs, csub = tid % cs, per = kChunk / cs;

    // the diagonal blocks start at zero; each slot subtracts its block below
    for (int x = tid; x < p.nqz * nw * 9; x += kPiThreads) {
        const int q = x / (nw * 9), ww = (x / 9) % nw, ij = x % 9;
        std_(Pi + ((((size_t)q * nw + ww) * p.na + a) * nb1 + p.nb) * 9 + ij, make_double2(0.0, 0.0));
    }
    for (int slot = 0; slot < p.nb; ++slot) {
        const int b = __ldg(p.neigh + (size_t)a * p.nb + slot);
        if (b < 0 || !SSE_BC(b, p.na, p.status)) {
            for (int x = tid; x < p.nqz * nw * 9; x += kPiThreads) {
                const int q = x / (nw * 9), ww = (x / 9) % nw, ij = x % 9;
                std_(Pi + ((((size_t)q * nw + ww) * p.na + a) * nb1 + slot) * 9 + ij, make_double2(0.0, 0.0));
            }
            continue;
        }
        __syncthreads();
        for (int x = tid; x < 3 * 144; x += kPiThreads) s_dh[x] = ldd(dH + ((size_t)a * p.nb + slot) * 3 * 144 + x);
        for (int q = 0; q < p.nqz; ++q) {
            double2 acc[9];
#pragma unroll
            for (int ij = 0; ij < 9; ++ij) acc[ij] = make_double2(0.0, 0.0);
            for (int k = 0; k < p.nkz; ++k) {
                const int kq = (k + q) % p.nkz;
                for (int m = 0; m < 144 / kChunk; ++m) {
                    // V_i rows E' = E + omega_first .. E + omega_max live at ring slot E' mod nw.
                    // Step E = -nw .. ne - 1: the steps E < 0 only fill the ring.
                    for (int E = -nw; E < p.ne; ++E) {
                        const int ep = E + omega_max;  // the V row formed at this step
                        __syncthreads();               // the previous step's reads are done
                        for (int x = tid; x < 288; x += kPiThreads) {
                            if (x < 144) {
                                if (ep >= 0 && ep < p.ne)
                                    s_ga[x] = ldd(Ga + (((size_t)kq * p.ne + ep) * p.na + a) * 144 + x);
                            } else if (E >= 0) {
                                s_gb[x - 144] = ldd(Gb + (((size_t)k * p.ne + E) * p.na + b) * 144 + (x - 144));
                            }
                        }
                        __syncthreads();
                        // V_i[r, s] = sum_u conj(dH_i[u, r]) Ga[u, s] and U_j^T[r, s] = U_j[s, r] =
                        // sum_v dH_j[s, v] Gb[v, r], for the chunk's channels (r, s)
                        for (int x = tid; x < 6 * kChunk; x += kPiThreads) {
                            const int which = x / (3 * kChunk), dir = (x / kChunk) % 3, cc = x % kChunk;
                            const int r = 4 * m + cc / 12, s = cc % 12;
                            double2 v = make_double2(0.0, 0.0);
                            if (which == 0) {
                                if (ep >= 0 && ep < p.ne) {
#pragma unroll
                                    for (int u = 0; u < 12; ++u) cmac_cj(v, s_dh[dir * 144 + u * 12 + r], s_ga[u * 12 + s]);
                                }
                                s_ring[((size_t)((ep % nw + nw) % nw) * 3 + dir) * kChunk + cc] = v;
                            } else if (E >= 0) {
#pragma unroll
                                for (int vv = 0; vv < 12; ++vv) cmac(v, s_dh[dir * 144 + s * 12 + vv], s_gb[vv * 12 + r]);
                                s_u[dir * kChunk + cc] = v;
                            }
                        }
                        __syncthreads();
                        if (E < 0 || !worker) continue;
                        const int epw = E + p.omega_first + w;  // this thread's V row
                        if (epw < 0 || epw >= p.ne) continue;   // E + omega off the grid
                        const double2 *vr = s_ring + (size_t)(epw % nw) * 3 * kChunk;
                        for (int c = csub * per; c < (csub + 1) * per; ++c) {
                            double2 vi[3], uj[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                vi[d] = vr[d * kChunk + c];
                                uj[d] = s_u[d * kChunk + c];
                            }
#pragma unroll
                            for (int i = 0; i < 3; ++i)
#pragma unroll
                                for (int j = 0; j < 3; ++j) cmac(acc[i * 3 + j], vi[i], uj[j]);
                        }
                    }
                }
            }
            // reduce over the channel subsets; one thread per w writes the block and updates
            // the diagonal (the same thread every slot, so the updates are ordered)
            __syncthreads();
            if (worker) {
#pragma unroll
                for (int ij = 0; ij < 9; ++ij) s_red[(size_t)tid * 9 + ij] = acc[ij];
            }
            __syncthreads();
            if (worker && csub == 0) {
                for (int ij = 0; ij < 9; ++ij) {
                    double2 t = make_double2(0.0, 0.0);
                    for (int c2 = 0; c2 < cs; ++c2) {
                        const double2 v = s_red[(size_t)(w * cs + c2) * 9 + ij];
                        t.x += v.x;
                        t.y += v.y;
                    }
                    const size_t base = (((size_t)q * nw + w) * p.na + a) * nb1;
                    std_(Pi + (base + slot) * 9 + ij, t);
                    double2 dg = ldd(Pi + (base + p.nb) * 9 + ij);
                    dg.x -= t.x;
                    dg.y -= t.y;
                    std_(Pi + (base + p.nb) * 9 + ij, dg);
                }
            }
        }
    }
}

}  // namespace

// Pi of the requested signs for the plan's geometry: (G_gt, G_lt) both required (each sign
// pairs one with the other); Pi_x [nqz][nw][na][nb + 1][3][3] in the plan's dtype.
sse_status launch_pi(const Plan &pl, const void *G_gt, const void *G_lt, void *Pi_gt, void *Pi_lt, cudaStream_t st) {
    const Dims &d = pl.d;
    PiArgs a{};
    int ns = 0;
    if (Pi_gt) {
        a.Ga[ns] = G_gt;
        a.Gb[ns] = G_lt;
        a.Pi[ns++] = Pi_gt;
    }
    if (Pi_lt) {
        a.Ga[ns] = G_lt;
        a.Gb[ns] = G_gt;
        a.Pi[ns++] = Pi_lt;
    }
    if (ns == 0) return SSE_OK;
    if (d.nw > kPiThreads) return set_error("the phonon self-energy kernel supports nw <= %d", kPiThreads), SSE_E_INVALID_ARG;
    int cs = 1;
    for (int c = kChunk; c >= 1; --c)
        if (kChunk % c == 0 && c * d.nw <= kPiThreads) {
            cs = c;
            break;
        }
    const size_t smem = (size_t)(3 * 144 + 144 + 144 + 3 * kChunk + d.nw * cs * 9 + (size_t)d.nw * 3 * kChunk) * 16;
    if (smem > 232448) return set_error("the phonon self-energy kernel: nw = %d needs too much shared memory", d.nw), SSE_E_INVALID_ARG;
    a.neigh = pl.geo.neigh;
    a.dH = pl.geo.dH;
    a.nkz = d.nkz;
    a.nqz = d.nqz;
    a.ne = d.ne;
    a.nw = d.nw;
    a.na = d.na;
    a.nb = d.nb;
    a.omega_first = d.omega_first;
    a.cs = cs;
    a.status = pl.d_status;
    dim3 grid((unsigned)d.na, (unsigned)ns);
    cudaError_t e;
    if (pl.geo.dtype == SSE_C128) {
        e = cudaFuncSetAttribute(sse_pi_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) sse_pi_kernel<double2><<<grid, kPiThreads, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(sse_pi_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) sse_pi_kernel<float2><<<grid, kPiThreads, smem, st>>>(a);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch sse_pi_kernel");
    return SSE_OK;
}

}  // namespace sse
