// The steps on either side of the self-energy kernels:
//  - the pre-combination of the phonon Green's function that Eq. 3 brackets,
//      Dt[q, w, a, slot] = D_ba - D_bb - D_aa + D_ab,  b = neigh[a, slot],
//    from the full phonon tensor [nqz][nw][na][nb + 1][3][3] of Section 2 (block nb of an
//    atom is its diagonal D_aa), done before the Sigma kernel per the input list of
//    Section 3 ("Dataflow Optimizations");
//  - the retarded component from the lesser and greater ones (Section 2, after Eq. 5),
//      Sigma^R = (Sigma^> - Sigma^<) / 2.
// Both are elementwise and bound by HBM bandwidth: grid-stride loops over 16-byte (or
// 8-byte) complex elements, with grids of a few CTAs per SM.  sse_execute_full chains them
// with the self-energy; there the mixed-mode kernels form Dt where they read it, so the
// pre-combined tensor is never stored.
#include <cuda_runtime.h>

#include "sse_internal.h"
#include "tc_ptx.h"

namespace sse {
namespace {

template <typename CT>
__device__ __forceinline__ double2 widen(CT v);
template <>
__device__ __forceinline__ double2 widen<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ double2 widen<float2>(float2 v) { return make_double2(tc::f32_to_f64(v.x), tc::f32_to_f64(v.y)); }
template <typename CT>
__device__ __forceinline__ CT narrow(double2 v);
template <>
__device__ __forceinline__ double2 narrow<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 narrow<float2>(double2 v) { return make_float2(tc::f64_to_f32(v.x), tc::f64_to_f32(v.y)); }

// One thread per Dt value (q, w, a, slot, ij); FP64 sum in the order ((D_ba - D_bb) - D_aa) + D_ab,
// rounded once to the storage type (the value the mixed kernels form on the fly).
template <typename CT>
__global__ void __launch_bounds__(256) sse_dtilde_kernel(const CT *__restrict__ D, const int32_t *__restrict__ neigh,
                                                         const int32_t *__restrict__ rev, CT *__restrict__ Dt,
                                                         long long n, int na, int nb, int32_t *status) {
    const size_t nb1 = (size_t)nb + 1;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const int ij = (int)(x % 9);
        const long long t = x / 9;
        const int slot = (int)(t % nb);
        const long long qa = t / nb;  // (q, w, a)
        const int a = (int)(qa % na);
        const size_t qw = (size_t)(qa / na) * na;
        const int f = __ldg(neigh + (size_t)a * nb + slot);
        double2 v = make_double2(0.0, 0.0);
        if (f >= 0 && SSE_BC(f, na, status) && SSE_BC(__ldg(rev + (size_t)a * nb + slot), nb, status)) {
            const int r = __ldg(rev + (size_t)a * nb + slot);
            const double2 ab = widen(D[((qw + a) * nb1 + slot) * 9 + ij]), aa = widen(D[((qw + a) * nb1 + nb) * 9 + ij]);
            const double2 ba = widen(D[((qw + f) * nb1 + r) * 9 + ij]), bb = widen(D[((qw + f) * nb1 + nb) * 9 + ij]);
            v.x = ((ba.x - bb.x) - aa.x) + ab.x;
            v.y = ((ba.y - bb.y) - aa.y) + ab.y;
        }
        Dt[x] = narrow<CT>(v);
    }
}

// Sigma^R = (Sigma^> - Sigma^<) / 2 over n complex values (exact scaling by one half).
template <typename CT>
__global__ void __launch_bounds__(256) sse_retarded_kernel(const CT *__restrict__ gt, const CT *__restrict__ lt,
                                                           CT *__restrict__ r, long long n) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const CT g = gt[x], l = lt[x];
        CT o;
        o.x = (g.x - l.x) * 0.5f;
        o.y = (g.y - l.y) * 0.5f;
        r[x] = o;
    }
}

unsigned grid_for(long long n, int device) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const long long want = (n + 255) / 256;
    const long long cap = 8LL * sms;  // 8 CTAs of 256 threads per SM: enough loads in flight
    return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

sse_status launch_dtilde(const Plan &p, const void *D, void *dt, cudaStream_t st) {
    if (!p.rev_ok) {
        set_error("the pre-combination needs every bond's reverse: some neigh[a][slot] = b has no slot of b holding a");
        return SSE_E_INVALID_ARG;
    }
    const long long n = (long long)d_elems(p.d);
    if (n == 0) return SSE_OK;
    const unsigned grid = grid_for(n, p.device);
    if (p.geo.dtype == SSE_C128)
        sse_dtilde_kernel<double2><<<grid, 256, 0, st>>>((const double2 *)D, p.geo.neigh, p.d_rev, (double2 *)dt, n,
                                                         p.d.na, p.d.nb, p.d_status);
    else
        sse_dtilde_kernel<float2><<<grid, 256, 0, st>>>((const float2 *)D, p.geo.neigh, p.d_rev, (float2 *)dt, n,
                                                        p.d.na, p.d.nb, p.d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch sse_dtilde_kernel");
    return SSE_OK;
}

sse_status launch_retarded(const Plan &p, const void *S_gt, const void *S_lt, void *S_r, cudaStream_t st) {
    const long long n = (long long)g_elems(p.d);
    if (n == 0) return SSE_OK;
    const unsigned grid = grid_for(n, p.device);
    if (p.geo.dtype == SSE_C128)
        sse_retarded_kernel<double2><<<grid, 256, 0, st>>>((const double2 *)S_gt, (const double2 *)S_lt, (double2 *)S_r, n);
    else
        sse_retarded_kernel<float2><<<grid, 256, 0, st>>>((const float2 *)S_gt, (const float2 *)S_lt, (float2 *)S_r, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch sse_retarded_kernel");
    return SSE_OK;
}

}  // namespace sse
