"""Pins for the CPU FP64 oracle of Eq. 3, against things other than itself.

Each pin is chosen so that a plausible slip in the oracle fails at least one:
  * hand-worked scalar example (golden file)     -> k wrap, E offset, conj, i/j order, neighbour
  * physics form with whole (NA*Norb)^2 matrices  -> the whole definition, Norb > 1, transposes
  * Nqz = Nw = 1 closed form with library matmul  -> E - omega_first offset, slot handling
  * anti-Hermiticity invariant                    -> product order and conjugate transposes
  * Norb = 1 scalar case vs numpy.convolve / roll -> Toeplitz-in-E and circular-in-k indexing
  * linearity, delta Dt, zero Dt                  -> dropped / doubled terms, (q, w, i, j) indexing
  * equivariance under k roll, E shift, slot permutation, empty and duplicate slots
"""
import os

import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def small_instance(nkz=3, nqz=2, ne=9, nw=3, na=5, nb=2, norb=2, seed=11, neigh=None, omega_first=1):
    geo = inputs.Geometry(nkz=nkz, nqz=nqz, ne=ne, nw=nw, na=na, nb=nb, norb=norb,
                          omega_first=omega_first)
    if neigh is None:
        offs = [1, -1, 2, -2][:nb]
        neigh = inputs.chain_neighbours(na, offs)
    return inputs.make_instance(geo, seed, neigh=neigh, hermitian_pairs=False)


def both(inst, sign="gt", omega_first=1):
    G, D = inst["G_" + sign], inst["D_" + sign]
    full = oracle.sigma_atoms(G, D, inst["dH"], inst["neigh"], omega_first=omega_first)
    nkz, ne, na = G.shape[:3]
    pts = [(k, e, a) for k in range(nkz) for e in range(ne) for a in range(na)]
    per_pt = oracle.sigma_points(G, D, inst["dH"], inst["neigh"], pts, omega_first=omega_first)
    per_pt = per_pt.reshape(nkz, ne, na, *per_pt.shape[1:])
    return full, per_pt


# --- hand-worked example ---------------------------------------------------------------

def test_worked_example_by_hand():
    rows = np.loadtxt(os.path.join(GOLDEN, "worked_example_norb1.txt"))
    nkz, nqz, ne, nw, na, nb, norb = 2, 2, 3, 2, 2, 1, 1
    neigh = np.array([[1], [0]], dtype=np.int32)
    dH = np.zeros((na, nb, 3, 1, 1), complex)
    dH[0, 0, :, 0, 0] = [1, 2j, 0]
    dH[1, 0, :, 0, 0] = [0, 1, 1 + 1j]
    G = np.zeros((nkz, ne, na, 1, 1), complex)
    for k in range(nkz):
        for e in range(ne):
            for b in range(na):
                G[k, e, b, 0, 0] = (1 + b) * (e + 1) + 10 * k
    D = np.zeros((nqz, nw, na, nb, 3, 3), complex)
    D[0, 0, 0, 0, 0, 1] = 1
    D[1, 1, 0, 0, 1, 0] = 2
    D[1, 0, 1, 0, 2, 1] = 1j
    S = oracle.sigma_atoms(G, D, dH, neigh)
    pts = rows[:, :3].astype(int)
    P = oracle.sigma_points(G, D, dH, neigh, pts)
    for (k, e, a, re, im), p in zip(rows, P):
        expect = re + 1j * im
        assert S[int(k), int(e), int(a), 0, 0] == pytest.approx(expect, abs=1e-12)
        assert p[0, 0] == pytest.approx(expect, abs=1e-12)


# --- brute force in the physics form ----------------------------------------------------

def physics_form(inst, sign="gt", omega_first=1):
    """Eq. 3 with whole matrices: Sigma_aa = [W_ij . Gdiag . H_j]_aa, where W_ij carries
    Dt_ij(q,w,a,b) * grad_i H_ab in block (a,b), H_j carries grad_j H_ba = (grad_j H_ab)^+
    in block (b,a), and Gdiag is block-diagonal in the atoms.  Needs distinct neighbours."""
    G, D, dH, neigh = inst["G_" + sign], inst["D_" + sign], inst["dH"], inst["neigh"]
    nkz, ne, na, n, _ = G.shape
    nqz, nw = D.shape[:2]
    nb = neigh.shape[1]
    N = na * n
    out = np.zeros((nkz, ne, na, n, n), complex)
    Hj = np.zeros((3, N, N), complex)
    for a in range(na):
        for s in range(nb):
            f = neigh[a, s]
            if f >= 0:
                for j in range(3):
                    Hj[j, f * n:(f + 1) * n, a * n:(a + 1) * n] = dH[a, s, j].conj().T
    for k in range(nkz):
        for e in range(ne):
            acc = np.zeros((N, N), complex)
            for q in range(nqz):
                for w in range(nw):
                    ep = e - (w + omega_first)
                    if ep < 0 or ep >= ne:
                        continue
                    Gd = np.zeros((N, N), complex)
                    for b in range(na):
                        Gd[b * n:(b + 1) * n, b * n:(b + 1) * n] = G[(k - q) % nkz, ep, b]
                    for i in range(3):
                        for j in range(3):
                            W = np.zeros((N, N), complex)
                            for a in range(na):
                                for s in range(nb):
                                    f = neigh[a, s]
                                    if f >= 0:
                                        W[a * n:(a + 1) * n, f * n:(f + 1) * n] += D[q, w, a, s, i, j] * dH[a, s, i]
                            acc += W @ Gd @ Hj[j]
            for a in range(na):
                out[k, e, a] = acc[a * n:(a + 1) * n, a * n:(a + 1) * n]
    return out


@pytest.mark.parametrize("norb", [1, 2, 3])
def test_brute_force_physics_form(norb):
    inst = small_instance(nkz=3, nqz=2, ne=7, nw=3, na=5, nb=2, norb=norb, seed=3 + norb)
    ref = physics_form(inst)
    full, pp = both(inst)
    assert rel(full, ref) < 1e-13
    assert rel(pp, ref) < 1e-13


def test_brute_force_norb12_few_points():
    inst = small_instance(nkz=2, nqz=2, ne=5, nw=2, na=4, nb=2, norb=12, seed=5)
    ref = physics_form(inst)
    full, pp = both(inst)
    assert rel(full, ref) < 1e-13 and rel(pp, ref) < 1e-13


def test_nqz_differs_from_nkz():
    inst = small_instance(nkz=3, nqz=5, ne=6, nw=2, na=4, nb=2, norb=2, seed=8)
    ref = physics_form(inst)
    full, pp = both(inst)
    assert rel(full, ref) < 1e-13 and rel(pp, ref) < 1e-13


def test_omega_first_zero_two_and_two_sided():
    """omega_first = 0 and 2, and negative omega_first: a frequency grid spanning both signs,
    so Sigma(E) gathers G(E - hbar omega) and G(E + hbar omega) (the two-sided exchange of
    Section 3, "Communication Avoidance")."""
    for of in (0, 2, -2, -4):
        inst = small_instance(nkz=2, nqz=2, ne=6, nw=3, na=4, nb=2, norb=2, seed=9 + of)
        ref = physics_form(inst, omega_first=of)
        full, pp = both(inst, omega_first=of)
        assert rel(full, ref) < 1e-13 and rel(pp, ref) < 1e-13


# --- closed form at Nqz = Nw = 1 ----------------------------------------------------------

def test_closed_form_single_frequency():
    inst = small_instance(nkz=3, nqz=1, ne=6, nw=1, na=6, nb=2, norb=12, seed=21)
    G, D, dH, neigh = inst["G_gt"], inst["D_gt"], inst["dH"], inst["neigh"]
    full, pp = both(inst)
    expect = np.zeros_like(full)
    for k in range(3):
        for e in range(1, 6):
            for a in range(6):
                for s in range(2):
                    f = neigh[a, s]
                    for i in range(3):
                        for j in range(3):
                            expect[k, e, a] += D[0, 0, a, s, i, j] * np.matmul(
                                np.matmul(dH[a, s, i], G[k, e - 1, f]), dH[a, s, j].conj().T)
    assert np.all(full[:, 0] == 0)
    assert rel(full, expect) < 1e-13 and rel(pp, expect) < 1e-13


# --- anti-Hermiticity invariant -------------------------------------------------------------

def test_anti_hermitian_invariant_tiny_config():
    inst = inputs.make_instance(inputs.TINY, 0)
    for sign in ("gt", "lt"):
        S = oracle.sigma_atoms(inst["G_" + sign], inst["D_" + sign], inst["dH"], inst["neigh"])
        assert np.linalg.norm(S) > 0
        assert rel(S, -np.conj(np.swapaxes(S, -1, -2))) < 1e-14


def test_anti_hermiticity_breaks_without_hermitian_dt():
    # Negative control: the invariant is not automatic -- a non-Hermitian Dt breaks it.
    inst = small_instance(nkz=2, nqz=2, ne=6, nw=2, na=4, nb=2, norb=4, seed=31)
    D = inst["D_gt"].copy()
    D[..., 0, 1] += 0.5
    S = oracle.sigma_atoms(inst["G_gt"], D, inst["dH"], inst["neigh"])
    assert rel(S, -np.conj(np.swapaxes(S, -1, -2))) > 1e-3


# --- scalar case against numpy.convolve and numpy.roll -----------------------------------------

def test_scalar_correlation_matches_convolve():
    rng = np.random.default_rng(7)
    nkz, nqz, ne, nw, na, of = 4, 3, 20, 5, 3, 1
    neigh = np.array([[2], [0], [1]], dtype=np.int32)
    G = (rng.standard_normal((nkz, ne, na, 1, 1)) + 1j * rng.standard_normal((nkz, ne, na, 1, 1)))
    dH = np.zeros((na, 1, 3, 1, 1), complex)
    dH[:, 0, 0, 0, 0] = rng.standard_normal(na) + 1j * rng.standard_normal(na)
    dH[:, 0, 1:, 0, 0] = rng.standard_normal((na, 2))  # unused: Dt is zero for i, j > 0
    D = np.zeros((nqz, nw, na, 1, 3, 3), complex)
    D[..., 0, 0, 0] = rng.standard_normal((nqz, nw, na)) + 1j * rng.standard_normal((nqz, nw, na))
    S = oracle.sigma_atoms(G, D, dH, neigh)
    for a in range(na):
        f = neigh[a, 0]
        expect = np.zeros((nkz, ne), complex)
        for q in range(nqz):
            filt = np.zeros(of + nw, complex)
            filt[of:] = D[q, :, a, 0, 0, 0]
            Gq = np.roll(G[:, :, f, 0, 0], shift=q, axis=0)  # Gq[k] = G[(k - q) mod nkz]
            for k in range(nkz):
                expect[k] += np.convolve(Gq[k], filt)[:ne]
        expect *= abs(dH[a, 0, 0, 0, 0]) ** 2
        assert rel(S[:, :, a, 0, 0], expect) < 1e-13


def test_two_sided_scalar_case_matches_convolve():
    """Norb = 1, Nkz = Nqz = 1, frequencies omega_w = w + omega_first from -m to nw - 1 - m:
    Sigma[E] = sum_w Dt[w] G[E - omega_w], a full convolution read m samples later."""
    rng = np.random.default_rng(8)
    ne, nw = 15, 7
    neigh = np.array([[0]], dtype=np.int32)
    G = rng.standard_normal((1, ne, 1, 1, 1)) + 1j * rng.standard_normal((1, ne, 1, 1, 1))
    dH = np.ones((1, 1, 3, 1, 1), complex)
    D = np.zeros((1, nw, 1, 1, 3, 3), complex)
    D[0, :, 0, 0, 0, 0] = rng.standard_normal(nw) + 1j * rng.standard_normal(nw)
    for m in (1, 3, 6, 9):
        S = oracle.sigma_atoms(G, D, dH, neigh, omega_first=-m)
        full = np.convolve(G[0, :, 0, 0, 0], D[0, :, 0, 0, 0, 0])
        expect = np.zeros(ne, complex)
        for e in range(ne):
            if 0 <= e + m < full.size:
                expect[e] = full[e + m]
        assert rel(S[0, :, 0, 0, 0], expect) < 1e-13, m


# --- linearity, zero and delta Dt ---------------------------------------------------------------

def test_linearity_in_G_and_Dt():
    i1 = small_instance(seed=41, norb=3)
    i2 = small_instance(seed=42, norb=3)
    dH, neigh = i1["dH"], i1["neigh"]
    alpha, beta = 0.7 - 0.2j, -1.3 + 0.5j
    S1 = oracle.sigma_atoms(i1["G_gt"], i1["D_gt"], dH, neigh)
    S2 = oracle.sigma_atoms(i2["G_gt"], i1["D_gt"], dH, neigh)
    S12 = oracle.sigma_atoms(alpha * i1["G_gt"] + beta * i2["G_gt"], i1["D_gt"], dH, neigh)
    assert rel(S12, alpha * S1 + beta * S2) < 1e-13
    T2 = oracle.sigma_atoms(i1["G_gt"], i2["D_gt"], dH, neigh)
    T12 = oracle.sigma_atoms(i1["G_gt"], alpha * i1["D_gt"] + beta * i2["D_gt"], dH, neigh)
    assert rel(T12, alpha * S1 + beta * T2) < 1e-13
    Z = oracle.sigma_atoms(i1["G_gt"], 0 * i1["D_gt"], dH, neigh)
    assert np.all(Z == 0)


@pytest.mark.parametrize("q0,w0,i0,j0", [(0, 0, 0, 0), (1, 2, 0, 2), (1, 1, 2, 1), (0, 2, 1, 0)])
def test_delta_dt_isolates_one_term(q0, w0, i0, j0):
    inst = small_instance(nkz=3, nqz=2, ne=8, nw=3, na=5, nb=2, norb=3, seed=51)
    G, dH, neigh = inst["G_gt"], inst["dH"], inst["neigh"]
    a0, s0 = 2, 1
    D = np.zeros_like(inst["D_gt"])
    D[q0, w0, a0, s0, i0, j0] = 1.0
    S = oracle.sigma_atoms(G, D, dH, neigh)
    f = neigh[a0, s0]
    expect = np.zeros_like(S)
    for k in range(3):
        for e in range(8):
            ep = e - (w0 + 1)
            if ep >= 0:
                expect[k, e, a0] = dH[a0, s0, i0] @ G[(k - q0) % 3, ep, f] @ dH[a0, s0, j0].conj().T
    assert rel(S, expect) < 1e-13


# --- equivariance and slot bookkeeping ---------------------------------------------------------

def test_k_roll_equivariance():
    inst = small_instance(seed=61, norb=2, nkz=4, nqz=3)
    S = oracle.sigma_atoms(inst["G_gt"], inst["D_gt"], inst["dH"], inst["neigh"])
    Sr = oracle.sigma_atoms(np.roll(inst["G_gt"], 1, axis=0), inst["D_gt"], inst["dH"], inst["neigh"])
    assert rel(Sr, np.roll(S, 1, axis=0)) < 1e-13


def test_energy_shift_equivariance():
    inst = small_instance(seed=62, norb=2, ne=10)
    G = inst["G_gt"]
    sh = 3
    Gs = np.zeros_like(G)
    Gs[:, sh:] = G[:, :-sh]
    S = oracle.sigma_atoms(G, inst["D_gt"], inst["dH"], inst["neigh"])
    Ss = oracle.sigma_atoms(Gs, inst["D_gt"], inst["dH"], inst["neigh"])
    assert rel(Ss[:, sh:], S[:, :-sh]) < 1e-13
    assert np.all(Ss[:, :sh] == 0)


def test_slot_permutation_invariance():
    inst = small_instance(seed=63, norb=2, nb=3, na=6)
    perm = np.array([2, 0, 1])
    S = oracle.sigma_atoms(inst["G_gt"], inst["D_gt"], inst["dH"], inst["neigh"])
    Sp = oracle.sigma_atoms(inst["G_gt"], inst["D_gt"][:, :, :, perm], inst["dH"][:, perm],
                            inst["neigh"][:, perm])
    assert rel(Sp, S) < 1e-13


def test_empty_slot_equals_zero_dt():
    inst = small_instance(seed=64, norb=2, nb=3, na=6)
    neigh = inst["neigh"].copy()
    neigh[2, 1] = -1
    neigh[4, 0] = -1
    D = inst["D_gt"].copy()
    D[:, :, 2, 1] = 0
    D[:, :, 4, 0] = 0
    S_empty = oracle.sigma_atoms(inst["G_gt"], inst["D_gt"], inst["dH"], neigh)
    S_zero = oracle.sigma_atoms(inst["G_gt"], D, inst["dH"], inst["neigh"])
    assert rel(S_empty, S_zero) < 1e-14


def test_duplicate_slot_doubles():
    inst = small_instance(seed=65, norb=2, nb=2, na=5)
    neigh = inst["neigh"].copy()
    neigh[:, 1] = -1
    S1 = oracle.sigma_atoms(inst["G_gt"], inst["D_gt"], inst["dH"], neigh)
    dup_n = np.repeat(neigh[:, :1], 2, axis=1)
    dup_h = np.repeat(inst["dH"][:, :1], 2, axis=1)
    dup_d = np.repeat(inst["D_gt"][:, :, :, :1], 2, axis=3)
    S2 = oracle.sigma_atoms(inst["G_gt"], dup_d, dup_h, dup_n)
    assert rel(S2, 2 * S1) < 1e-14


def test_points_entry_matches_atoms_entry_tiny():
    inst = inputs.make_instance(inputs.TINY, 0)
    S = oracle.sigma_atoms(inst["G_lt"], inst["D_lt"], inst["dH"], inst["neigh"], 3, 9)
    pts = [(k, e, a) for k in range(3) for e in (0, 1, 4, 5, 30, 47) for a in (3, 8)]
    P = oracle.sigma_points(inst["G_lt"], inst["D_lt"], inst["dH"], inst["neigh"], pts)
    ref = np.stack([S[k, e, a - 3] for k, e, a in pts])
    assert rel(P, ref) < 1e-14


def test_oracle_rejects_bad_neighbour():
    inst = small_instance(seed=66)
    neigh = inst["neigh"].copy()
    neigh[0, 0] = 99
    with pytest.raises(ValueError):
        oracle.sigma_atoms(inst["G_gt"], inst["D_gt"], inst["dH"], neigh)
