/*
 * CPU FP64 oracle for the electron scattering self-energy Sigma^{<>} (Eq. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code: only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes (Eq. 3, Section 2, read discretely as in the Sigma listing of
 * Section 3): for every output point (kz, E, a) and each sign separately
 *
 *   Sigma[k,E,a] = sum_{slot : f = neigh[a,slot] >= 0} sum_{i,j in x,y,z}
 *                  sum_{q < Nqz} sum_{w < Nw, E' = E - (w + omega_first) >= 0}
 *                  Dt[q,w,a,slot,i,j] * dH[a,slot,i] . G[(k - q) mod Nkz, E', f] . dH[a,slot,j]^dagger
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - the prefactor i and the frequency weight d(hbar w)/2pi of Eq. 3 are left to the
 *    caller (factor 1);
 *  - the undefined index l of Eq. 3's sum is read as the neighbour b;
 *  - the reverse bond block grad_j H_ba is the conjugate transpose of the stored
 *    forward block dH[a,slot,j] (the listing's float64 dH is taken complex);
 *  - kz - qz wraps modulo Nkz (kz is periodic on [-pi, pi], Section 2);
 *  - the phonon frequency index w means (w + omega_first) energy-grid steps, and an
 *    energy E - omega off the grid contributes nothing (no wrap); omega_first may be
 *    negative, so one frequency grid can hold both E - hbar omega and E + hbar omega (the
 *    two-sided exchange G(E +- hbar omega) of Section 3, "Communication Avoidance");
 *  - Dt is the already pre-combined D_ba - D_bb - D_aa + D_ab (Section 3 input list);
 *  - Sigma is overwritten (accumulated into zero, the SCBA start value of Section 2).
 *
 * Entry points for Sigma:
 *  - oracle_sigma_points: the definition above, term by term, for chosen points;
 *  - oracle_sigma_atoms: the same sum after the paper's redundancy removal
 *    (Section 3, "Dataflow Optimizations": dH.G does not depend on (qz, w), so the
 *    product M_ij = dH_i . G . dH_j^dagger is formed once per (kz', E', a, b) and then
 *    correlated with Dt).  Exact rearrangement; agrees with the first to rounding.
 *
 * Complex values are C99 `double complex`; all arithmetic is FP64; no BLAS; the
 * summation order is slot, i, j, q, w ascending in both entry points.
 *
 * The steps on either side of Sigma: oracle_dtilde (the phonon pre-combination of Eq. 3)
 * and oracle_retarded (Sigma^R from Sigma^> and Sigma^<, Section 2).  The phonon
 * self-energy of Eqs. 4 and 5: oracle_pi.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define N3D 3

typedef double complex cplx;

/* Sizes of one instance; the symbols of Table 1. */
typedef struct {
    int32_t nkz, nqz, ne, nw, na, nb, norb, omega_first;
} oracle_geometry;

static size_t g_index(const oracle_geometry *g, int k, int e, int a) {
    /* G / Sigma block (k, E, a) in [nkz][ne][na][norb][norb] */
    return (((size_t)k * g->ne + e) * g->na + a) * (size_t)g->norb * g->norb;
}

static size_t dh_index(const oracle_geometry *g, int a, int slot, int i) {
    /* dH block (a, slot, i) in [na][nb][3][norb][norb] */
    return (((size_t)a * g->nb + slot) * N3D + i) * (size_t)g->norb * g->norb;
}

static size_t d_index(const oracle_geometry *g, int q, int w, int a, int slot, int i, int j) {
    /* Dt scalar (q, w, a, slot, i, j) in [nqz][nw][na][nb][3][3] */
    return ((((size_t)q * g->nw + w) * g->na + a) * g->nb + slot) * (N3D * N3D) + i * N3D + j;
}

/* c = a . b for n x n row-major blocks */
static void matmul(int n, const cplx *a, const cplx *b, cplx *c) {
    for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
            cplx acc = 0;
            for (int t = 0; t < n; ++t) acc += a[r * n + t] * b[t * n + s];
            c[r * n + s] = acc;
        }
}

/* c = a . b^dagger for n x n row-major blocks */
static void matmul_adj(int n, const cplx *a, const cplx *b, cplx *c) {
    for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
            cplx acc = 0;
            for (int t = 0; t < n; ++t) acc += a[r * n + t] * conj(b[s * n + t]);
            c[r * n + s] = acc;
        }
}

static int valid_geometry(const oracle_geometry *g) {
    return g && g->nkz > 0 && g->nqz > 0 && g->ne > 0 && g->nw > 0 && g->na > 0 &&
           g->nb > 0 && g->norb > 0 && g->omega_first > -(1 << 20) && g->omega_first < (1 << 20);
}

static int wrap_k(int k, int q, int nkz) {
    int r = (k - q) % nkz;
    return r < 0 ? r + nkz : r;
}

/*
 * Eq. 3 term by term for npts output points pts[p] = (k, E, a); out[p] is one
 * norb x norb block.  Returns 0, or -1 on a bad argument / neighbour index.
 */
int oracle_sigma_points(const oracle_geometry *g, const int32_t *neigh, const cplx *dH,
                        const cplx *G, const cplx *Dt, int64_t npts, const int32_t *pts,
                        cplx *out) {
    if (!valid_geometry(g) || !neigh || !dH || !G || !Dt || npts < 0 || (npts && (!pts || !out)))
        return -1;
    for (int64_t p = 0; p < (int64_t)g->na * g->nb; ++p)
        if (neigh[p] < -1 || neigh[p] >= g->na) return -1;
    for (int64_t p = 0; p < npts; ++p) {
        const int32_t *pt = pts + 3 * p;
        if (pt[0] < 0 || pt[0] >= g->nkz || pt[1] < 0 || pt[1] >= g->ne || pt[2] < 0 || pt[2] >= g->na)
            return -1;
    }
    const int n = g->norb, nn = n * n;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t p = 0; p < npts; ++p) {
        const int k = pts[3 * p], e = pts[3 * p + 1], a = pts[3 * p + 2];
        cplx *acc = out + (size_t)p * nn;
        cplx *x = malloc(sizeof(cplx) * nn), *m = malloc(sizeof(cplx) * nn);
        if (!x || !m) { bad |= 1; free(x); free(m); continue; }
        memset(acc, 0, sizeof(cplx) * nn);
        for (int slot = 0; slot < g->nb; ++slot) {
            const int f = neigh[(size_t)a * g->nb + slot];
            if (f < 0) continue; /* empty slot */
            for (int i = 0; i < N3D; ++i)
                for (int j = 0; j < N3D; ++j)
                    for (int q = 0; q < g->nqz; ++q)
                        for (int w = 0; w < g->nw; ++w) {
                            const int ep = e - (w + g->omega_first);
                            if (ep < 0 || ep >= g->ne) continue; /* E - omega off the energy grid */
                            const cplx d = Dt[d_index(g, q, w, a, slot, i, j)];
                            const cplx *gb = G + g_index(g, wrap_k(k, q, g->nkz), ep, f);
                            matmul(n, dH + dh_index(g, a, slot, i), gb, x);   /* dH_i . G       */
                            matmul_adj(n, x, dH + dh_index(g, a, slot, j), m); /* ... . dH_j^+ */
                            for (int r = 0; r < nn; ++r) acc[r] += d * m[r];
                        }
        }
        free(x);
        free(m);
    }
    return bad ? -1 : 0;
}

/*
 * All points of atoms [a_begin, a_end) after the redundancy removal of Section 3:
 * M_ij[k', E'] = dH_i . G[k', E', f] . dH_j^dagger once per (k', E', a, slot), then
 * Sigma[k, E, a] += sum_{i,j,q,w} Dt[q,w,a,slot,i,j] M_ij[(k-q) mod Nkz, E - omega_w].
 * out is [nkz][ne][a_end - a_begin][norb][norb].  Returns 0 or -1.
 */
int oracle_sigma_atoms(const oracle_geometry *g, const int32_t *neigh, const cplx *dH,
                       const cplx *G, const cplx *Dt, int32_t a_begin, int32_t a_end, cplx *out) {
    if (!valid_geometry(g) || !neigh || !dH || !G || !Dt || !out || a_begin < 0 ||
        a_end > g->na || a_begin > a_end)
        return -1;
    for (int64_t p = 0; p < (int64_t)g->na * g->nb; ++p)
        if (neigh[p] < -1 || neigh[p] >= g->na) return -1;
    const int n = g->norb, nn = n * n, nsl = a_end - a_begin;
    const size_t mblocks = (size_t)g->nkz * g->ne * N3D * N3D;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int a = a_begin; a < a_end; ++a) {
        cplx *M = malloc(sizeof(cplx) * nn * mblocks), *x = malloc(sizeof(cplx) * nn);
        if (!M || !x) { bad |= 1; free(M); free(x); continue; }
        for (int k = 0; k < g->nkz; ++k)
            for (int e = 0; e < g->ne; ++e)
                memset(out + (((size_t)k * g->ne + e) * nsl + (a - a_begin)) * nn, 0, sizeof(cplx) * nn);
        for (int slot = 0; slot < g->nb; ++slot) {
            const int f = neigh[(size_t)a * g->nb + slot];
            if (f < 0) continue;
            /* M_ij for every (k', E'): independent of (q, w) */
            for (int kp = 0; kp < g->nkz; ++kp)
                for (int ep = 0; ep < g->ne; ++ep)
                    for (int i = 0; i < N3D; ++i) {
                        matmul(n, dH + dh_index(g, a, slot, i), G + g_index(g, kp, ep, f), x);
                        for (int j = 0; j < N3D; ++j)
                            matmul_adj(n, x, dH + dh_index(g, a, slot, j),
                                       M + ((((size_t)kp * g->ne + ep) * N3D + i) * N3D + j) * nn);
                    }
            /* correlation over (q, w) */
            for (int k = 0; k < g->nkz; ++k)
                for (int e = 0; e < g->ne; ++e) {
                    cplx *acc = out + (((size_t)k * g->ne + e) * nsl + (a - a_begin)) * nn;
                    for (int i = 0; i < N3D; ++i)
                        for (int j = 0; j < N3D; ++j)
                            for (int q = 0; q < g->nqz; ++q)
                                for (int w = 0; w < g->nw; ++w) {
                                    const int ep = e - (w + g->omega_first);
                                    if (ep < 0 || ep >= g->ne) continue;
                                    const cplx d = Dt[d_index(g, q, w, a, slot, i, j)];
                                    const cplx *m = M + ((((size_t)wrap_k(k, q, g->nkz) * g->ne + ep) * N3D + i) * N3D + j) * nn;
                                    for (int r = 0; r < nn; ++r) acc[r] += d * m[r];
                                }
                }
        }
        free(M);
        free(x);
    }
    return bad ? -1 : 0;
}

/*
 * The pre-combination of the phonon Green's function that Eq. 3 brackets, done before the
 * Sigma kernel in Section 3 ("Dataflow Optimizations", the input list):
 *   Dt[q,w,a,slot,i,j] = D_ba - D_bb - D_aa + D_ab,   b = neigh[a,slot],
 * from the full phonon tensor D [nqz][nw][na][nb+1][3][3] of Section 2 (the shape with
 * NB + 1 blocks per atom).  Readings taken here:
 *  - block slot (< nb) of atom a is D_ab for b = neigh[a,slot]; block nb is the diagonal D_aa;
 *  - D_ba is the block of atom b at the first slot s' with neigh[b,s'] = a; a bond whose
 *    reverse is not listed makes the call fail (-1): Eq. 3 needs D_ba;
 *  - an empty slot (neigh = -1) gives Dt = 0;
 *  - the sum is taken in the order ((D_ba - D_bb) - D_aa) + D_ab.
 * Dt is [nqz][nw][na][nb][3][3].  Returns 0 or -1.
 */
int oracle_dtilde(const oracle_geometry *g, const int32_t *neigh, const cplx *D, cplx *Dt) {
    if (!valid_geometry(g) || !neigh || !D || !Dt) return -1;
    const int nb = g->nb, nb1 = g->nb + 1;
    for (int64_t p = 0; p < (int64_t)g->na * nb; ++p)
        if (neigh[p] < -1 || neigh[p] >= g->na) return -1;
    for (int a = 0; a < g->na; ++a)
        for (int slot = 0; slot < nb; ++slot) {
            const int b = neigh[(size_t)a * nb + slot];
            if (b < 0) continue;
            int rev = -1;
            for (int s2 = 0; s2 < nb && rev < 0; ++s2)
                if (neigh[(size_t)b * nb + s2] == a) rev = s2;
            if (rev < 0) return -1;
            for (int q = 0; q < g->nqz; ++q)
                for (int w = 0; w < g->nw; ++w) {
                    const size_t base = ((size_t)q * g->nw + w) * g->na;
                    const cplx *d_ab = D + ((base + a) * nb1 + slot) * (N3D * N3D);
                    const cplx *d_aa = D + ((base + a) * nb1 + nb) * (N3D * N3D);
                    const cplx *d_ba = D + ((base + b) * nb1 + rev) * (N3D * N3D);
                    const cplx *d_bb = D + ((base + b) * nb1 + nb) * (N3D * N3D);
                    cplx *out = Dt + ((base + a) * nb + slot) * (N3D * N3D);
                    for (int ij = 0; ij < N3D * N3D; ++ij)
                        out[ij] = ((d_ba[ij] - d_bb[ij]) - d_aa[ij]) + d_ab[ij];
                }
        }
    for (int a = 0; a < g->na; ++a)
        for (int slot = 0; slot < nb; ++slot) {
            if (neigh[(size_t)a * nb + slot] >= 0) continue;
            for (int q = 0; q < g->nqz; ++q)
                for (int w = 0; w < g->nw; ++w)
                    memset(Dt + ((((size_t)q * g->nw + w) * g->na + a) * nb + slot) * (N3D * N3D), 0,
                           sizeof(cplx) * N3D * N3D);
        }
    return 0;
}

/*
 * The retarded self-energy from the lesser and greater ones (Section 2, the relation
 * given after Eq. 5): Sigma^R = (Sigma^> - Sigma^<) / 2, elementwise over n complex values.
 */
int oracle_retarded(int64_t n, const cplx *S_gt, const cplx *S_lt, cplx *S_r) {
    if (n < 0 || (n && (!S_gt || !S_lt || !S_r))) return -1;
    for (int64_t x = 0; x < n; ++x) S_r[x] = (S_gt[x] - S_lt[x]) * 0.5;
    return 0;
}

/*
 * The phonon scattering self-energy Pi^s (Eq. 5 for the off-diagonal blocks, Eq. 4 for the
 * diagonal ones, Section 2), kept for the N_B neighbour couplings and the diagonal block
 * as Section 2 states, in the shape of the phonon Green's function:
 *   Pi [nqz][nw][na][nb + 1][3][3]   (block nb of an atom is its diagonal block).
 * For a neighbour slot with b = neigh[a,slot] >= 0 (Eq. 5):
 *   Pi[q,w,a,slot,i,j] = sum_{k < nkz} sum_{E : E' = E + (w + omega_first) < ne}
 *       tr{ dH[a,slot,i]^dagger . Ga[(k + q) mod nkz, E', a] . dH[a,slot,j] . Gb[k, E, b] }
 * and for the diagonal block (Eq. 4) the same trace summed over the neighbour slots with
 * the opposite sign:
 *   Pi[q,w,a,nb,i,j] = - sum_{slot : b >= 0} Pi[q,w,a,slot,i,j].
 * Readings taken here (also in the design notes):
 *  - the prefactors of Eqs. 4 and 5 (-i and +i) and the weight dE/2pi are left to the
 *    caller (factor 1), keeping their relative sign: the diagonal block is minus the sum;
 *  - Eq. 4's undefined sum index l is the neighbour b (as for Eq. 3);
 *  - grad_i H_ba is the conjugate transpose of the stored dH[a,slot,i], grad_j H_ab = dH[a,slot,j];
 *  - kz + qz wraps modulo nkz; E + omega above the energy grid contributes nothing;
 *  - for Pi^> the caller passes Ga = G^> and Gb = G^< (G^{<>}_aa paired with G^{><}_bb), and
 *    the reverse for Pi^<;
 *  - an empty slot gives a zero block and adds nothing to the diagonal.
 * The sums run k, E ascending; the diagonal block sums the slots ascending.  Returns 0 or -1.
 */
int oracle_pi(const oracle_geometry *g, const int32_t *neigh, const cplx *dH, const cplx *Ga, const cplx *Gb,
              cplx *Pi) {
    if (!valid_geometry(g) || !neigh || !dH || !Ga || !Gb || !Pi) return -1;
    for (int64_t p = 0; p < (int64_t)g->na * g->nb; ++p)
        if (neigh[p] < -1 || neigh[p] >= g->na) return -1;
    const int n = g->norb, nn = n * n, nb = g->nb, nb1 = g->nb + 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int a = 0; a < g->na; ++a) {
        cplx *x = malloc(sizeof(cplx) * nn), *y = malloc(sizeof(cplx) * nn), *hi = malloc(sizeof(cplx) * nn);
        if (!x || !y || !hi) { bad |= 1; free(x); free(y); free(hi); continue; }
        for (int q = 0; q < g->nqz; ++q)
            for (int w = 0; w < g->nw; ++w) {
                cplx *diag = Pi + ((((size_t)q * g->nw + w) * g->na + a) * nb1 + nb) * (N3D * N3D);
                for (int ij = 0; ij < N3D * N3D; ++ij) diag[ij] = 0;
                for (int slot = 0; slot < nb; ++slot) {
                    const int b = neigh[(size_t)a * nb + slot];
                    cplx *blk = Pi + ((((size_t)q * g->nw + w) * g->na + a) * nb1 + slot) * (N3D * N3D);
                    for (int i = 0; i < N3D; ++i)
                        for (int j = 0; j < N3D; ++j) {
                            cplx acc = 0;
                            if (b >= 0) {
                                const cplx *hI = dH + dh_index(g, a, slot, i), *hJ = dH + dh_index(g, a, slot, j);
                                for (int r = 0; r < n; ++r)
                                    for (int c = 0; c < n; ++c) hi[r * n + c] = conj(hI[c * n + r]); /* dH_i^dagger */
                                for (int k = 0; k < g->nkz; ++k)
                                    for (int e = 0; e < g->ne; ++e) {
                                        const int ep = e + w + g->omega_first;
                                        if (ep < 0 || ep >= g->ne) continue; /* E + omega off the energy grid */
                                        const int kq = (k + q) % g->nkz;
                                        matmul(n, hi, Ga + g_index(g, kq, ep, a), x);  /* dH_i^+ . Ga      */
                                        matmul(n, x, hJ, y);                            /* ... . dH_j       */
                                        const cplx *gb = Gb + g_index(g, k, e, b);
                                        for (int r = 0; r < n; ++r)                     /* tr{ ... . Gb }   */
                                            for (int c = 0; c < n; ++c) acc += y[r * n + c] * gb[c * n + r];
                                    }
                            }
                            blk[i * N3D + j] = acc;
                        }
                }
                for (int slot = 0; slot < nb; ++slot) {
                    if (neigh[(size_t)a * nb + slot] < 0) continue;
                    const cplx *blk = Pi + ((((size_t)q * g->nw + w) * g->na + a) * nb1 + slot) * (N3D * N3D);
                    for (int ij = 0; ij < N3D * N3D; ++ij) diag[ij] -= blk[ij];
                }
            }
        free(x);
        free(y);
        free(hi);
    }
    return bad ? -1 : 0;
}

/* Threads the OpenMP runtime will use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
