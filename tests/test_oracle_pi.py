"""Pins of the oracle's phonon self-energy Pi (Eq. 5 off-diagonal, Eq. 4 diagonal) on the
CPU: a hand-worked scalar case, a correlation against numpy.correlate, the momentum
direction, Hermiticity in (i, j), the diagonal-block relation and linearity."""
import os

import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pi_scalar.txt")


def scalar_case():
    nkz, ne, na = 2, 3, 2
    h = np.array([[1, 2, 3], [1, 1 + 1j, 1 + 2j]])
    dH = h.reshape(na, 1, 3, 1, 1).astype(complex)
    Ga = np.zeros((nkz, ne, na, 1, 1), complex)
    Gb = np.zeros((nkz, ne, na, 1, 1), complex)
    for k in range(nkz):
        for e in range(ne):
            Ga[k, e, 0] = 1 + k + 10 * e
            Ga[k, e, 1] = 1j * (e + 1)
            Gb[k, e, 0] = 2
            Gb[k, e, 1] = k + 1
    neigh = np.array([[1], [0]], np.int32)
    return Ga, Gb, dH, neigh


def test_hand_worked_scalar_case():
    Ga, Gb, dH, neigh = scalar_case()
    Pi = oracle.pi(Ga, Gb, dH, neigh, nqz=2, nw=1)
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 10
    for q, a, slot, i, j, re, im in rows:
        assert Pi[int(q), 0, int(a), int(slot), int(i), int(j)] == complex(float(re), float(im))


def test_scalar_correlation_matches_numpy():
    """Norb = 1, Nkz = 1, dH = 1: Pi(w) = sum_E Ga[E + omega_w] Gb[E], a cross-correlation."""
    rng = np.random.default_rng(1)
    ne, nw = 17, 6
    for of in (0, 1, 3, -2, -5):  # negative: E - |omega| as well (two-sided grid)
        x = rng.standard_normal(ne) + 1j * rng.standard_normal(ne)
        y = rng.standard_normal(ne) + 1j * rng.standard_normal(ne)
        Ga = np.zeros((1, ne, 2, 1, 1), complex)
        Gb = np.zeros((1, ne, 2, 1, 1), complex)
        Ga[0, :, 0, 0, 0] = x
        Gb[0, :, 1, 0, 0] = y
        dH = np.ones((2, 1, 3, 1, 1), complex)
        Pi = oracle.pi(Ga, Gb, dH, np.array([[1], [0]], np.int32), nqz=1, nw=nw, omega_first=of)
        c = np.correlate(x, np.conj(y), mode="full")  # c[lag + ne - 1] = sum_n x[n + lag] y[n]
        for w in range(nw):
            lag = w + of
            want = c[lag + ne - 1] if -ne < lag < ne else 0
            assert Pi[0, w, 0, 0, 0, 0] == pytest.approx(want, abs=1e-12)


def test_momentum_direction():
    """Ga only at k0 and Gb only at k1: Pi is nonzero only for q = (k0 - k1) mod Nkz (the
    pairing Ga(k + q) with Gb(k))."""
    rng = np.random.default_rng(2)
    nkz, ne, na = 5, 6, 3
    geo = inputs.Geometry(nkz=nkz, nqz=nkz, ne=ne, nw=2, na=na, nb=2, norb=2)
    neigh = np.array([[1, 2], [2, 0], [0, 1]], np.int32)
    inst = inputs.make_instance(geo, 3, neigh=neigh)
    for k0, k1 in ((3, 1), (0, 4)):
        Ga = np.zeros_like(inst["G_gt"])
        Gb = np.zeros_like(inst["G_lt"])
        Ga[k0] = inst["G_gt"][k0]
        Gb[k1] = inst["G_lt"][k1]
        Pi = oracle.pi(Ga, Gb, inst["dH"], neigh, nqz=nkz, nw=2)
        for q in range(nkz):
            nz = np.abs(Pi[q]).max()
            assert (nz > 1e-9) == (q == (k0 - k1) % nkz), (k0, k1, q)


def test_hermitian_in_ij_for_anti_hermitian_g_and_diagonal_relation():
    geo = inputs.Geometry(nkz=3, nqz=2, ne=9, nw=3, na=5, nb=3, norb=3)
    rng = np.random.default_rng(4)
    neigh = np.array([[1, 4, -1], [2, 0, 3], [3, 1, 1], [4, 2, 0], [0, 3, 2]], np.int32)
    inst = inputs.make_instance(geo, 5, neigh=neigh, hermitian_pairs=False)
    for Ga, Gb in ((inst["G_gt"], inst["G_lt"]), (inst["G_lt"], inst["G_gt"])):
        Pi = oracle.pi(Ga, Gb, inst["dH"], neigh, nqz=2, nw=3)
        np.testing.assert_allclose(Pi, np.conj(np.swapaxes(Pi, -1, -2)), atol=1e-10)
        valid = neigh >= 0
        diag = -np.sum(Pi[:, :, :, :3] * valid[None, None, :, :, None, None], axis=3)
        np.testing.assert_allclose(Pi[:, :, :, 3], diag, atol=1e-10)
        assert np.all(Pi[:, :, 0, 2] == 0)  # empty slot
    # a G that is not anti-Hermitian breaks the (i, j) symmetry (negative control)
    G2 = inst["G_gt"] + rng.standard_normal(inst["G_gt"].shape)
    Pi2 = oracle.pi(G2, inst["G_lt"], inst["dH"], neigh, nqz=2, nw=3)
    assert np.abs(Pi2 - np.conj(np.swapaxes(Pi2, -1, -2))).max() > 1e-3


def test_einsum_restatement_and_linearity():
    """The trace written as one einsum over all indices (no loops, no matmul chain), and
    linearity in each Green's function."""
    geo = inputs.Geometry(nkz=2, nqz=3, ne=7, nw=2, na=4, nb=2, norb=2)
    neigh = np.array([[1, 3], [2, 0], [3, 1], [0, 2]], np.int32)
    inst = inputs.make_instance(geo, 6, neigh=neigh)
    Ga, Gb, dH = inst["G_gt"], inst["G_lt"], inst["dH"]
    Pi = oracle.pi(Ga, Gb, dH, neigh, nqz=3, nw=2)
    for q in range(3):
        for w in range(2):
            n = geo.ne - (w + 1)
            for a in range(4):
                for s in range(2):
                    b = neigh[a, s]
                    ga = Ga[(np.arange(2) + q) % 2][:, w + 1:w + 1 + n, a]  # [k, E, u, v]
                    gb = Gb[:, :n, b]
                    want = np.einsum("iur,kEuv,jvt,kEtr->ij", np.conj(dH[a, s]), ga, dH[a, s], gb)
                    np.testing.assert_allclose(Pi[q, w, a, s], want, atol=1e-10)
    Pi2 = oracle.pi(Ga + 2 * Gb, Gb, dH, neigh, nqz=3, nw=2)
    Pi3 = oracle.pi(Gb, Gb, dH, neigh, nqz=3, nw=2)
    np.testing.assert_allclose(Pi2, Pi + 2 * Pi3, atol=1e-10)
