"""Pins of the oracle's steps on either side of Sigma (no GPU): the pre-combination
Dt = D_ba - D_bb - D_aa + D_ab of Eq. 3 and the retarded relation of Section 2."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dtilde_ring3.txt")
P = [[1, 2, 3], [5, 7, 11], [13, 17, 19]]
Q = [[2, 3, 5], [7, 11, 13], [17, 19, 23]]
RING = np.array([[2, 1], [0, 2], [1, 0]], dtype=np.int32)


def ring_tensor():
    ij = np.subtract.outer(np.arange(3), np.arange(3))
    D = np.zeros((1, 1, 3, 3, 3, 3), dtype=np.complex128)
    for a in range(3):
        for s in range(3):
            D[0, 0, a, s] = P[a][s] + 1j * Q[a][s] * ij
    return D


def test_hand_worked_ring():
    Dt = oracle.dtilde(ring_tensor(), RING)
    ij = np.subtract.outer(np.arange(3), np.arange(3))
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for a, s, pd, qd in (map(int, r) for r in rows):
        np.testing.assert_array_equal(Dt[0, 0, a, s], pd + 1j * qd * ij)


def random_full(rng, nqz, nw, na, nb):
    x = rng.standard_normal((nqz, nw, na, nb + 1, 3, 3, 2))
    return x[..., 0] + 1j * x[..., 1]


def chain(na, offsets=(-2, -1, 1, 2)):
    a = np.arange(na)[:, None]
    return ((a + np.array(offsets)[None, :]) % na).astype(np.int32)


def test_symmetric_in_the_bond():
    """Dt_ab and Dt_ba are the same sum of four blocks."""
    rng = np.random.default_rng(1)
    neigh = chain(9)
    Dt = oracle.dtilde(random_full(rng, 2, 3, 9, 4), neigh)
    for a in range(9):
        for s in range(4):
            b = neigh[a, s]
            s2 = list(neigh[b]).index(a)
            # the same four blocks, summed in another order: equal to rounding
            np.testing.assert_allclose(Dt[:, :, a, s], Dt[:, :, b, s2], rtol=0, atol=1e-14)


def test_hermitian_blocks_give_hermitian_dtilde():
    """With D_ba^ij = conj(D_ab^ji) and Hermitian diagonal blocks, Dt is Hermitian in (i, j)
    -- the property the anti-Hermiticity invariant of Sigma needs."""
    rng = np.random.default_rng(2)
    na, nb = 7, 4
    neigh = chain(na)
    D = random_full(rng, 2, 2, na, nb)
    D[:, :, :, nb] = D[:, :, :, nb] + np.conj(np.swapaxes(D[:, :, :, nb], -1, -2))
    for a in range(na):
        for s in range(nb):
            b = neigh[a, s]
            s2 = list(neigh[b]).index(a)
            if (b, s2) > (a, s):
                D[:, :, b, s2] = np.conj(np.swapaxes(D[:, :, a, s], -1, -2))
    Dt = oracle.dtilde(D, neigh)
    np.testing.assert_allclose(Dt, np.conj(np.swapaxes(Dt, -1, -2)), rtol=0, atol=1e-13)
    # a non-Hermitian diagonal block breaks it (negative control)
    D[0, 0, 3, nb, 0, 1] += 1.0
    Dt2 = oracle.dtilde(D, neigh)
    assert np.abs(Dt2 - np.conj(np.swapaxes(Dt2, -1, -2))).max() > 0.5


def test_equal_blocks_cancel_and_empty_slots_are_zero():
    rng = np.random.default_rng(3)
    neigh = chain(6)
    neigh[2, 1] = -1
    neigh[neigh[2, 1] if neigh[2, 1] >= 0 else 1, 2] = -1  # its reverse bond (1 -> 2) too
    blk = rng.standard_normal((3, 3))
    D = np.broadcast_to(blk, (1, 2, 6, 5, 3, 3)).astype(np.complex128)
    Dt = oracle.dtilde(D, neigh)
    assert np.all(Dt == 0)
    D = random_full(rng, 1, 2, 6, 4)
    Dt = oracle.dtilde(D, neigh)
    assert np.all(Dt[:, :, 2, 1] == 0) and np.all(Dt[:, :, 1, 2] == 0)
    assert np.abs(Dt[:, :, 0, 0]).min() > 0


def test_bond_without_its_reverse_is_rejected():
    neigh = np.array([[1, -1], [-1, -1]], dtype=np.int32)  # 0 -> 1 but not 1 -> 0
    with pytest.raises(ValueError):
        oracle.dtilde(np.zeros((1, 1, 2, 3, 3, 3), complex), neigh)


def test_linear_in_d():
    rng = np.random.default_rng(4)
    neigh = chain(8)
    A, B = random_full(rng, 2, 2, 8, 4), random_full(rng, 2, 2, 8, 4)
    np.testing.assert_allclose(oracle.dtilde(A + 2.5 * B, neigh),
                               oracle.dtilde(A, neigh) + 2.5 * oracle.dtilde(B, neigh), atol=1e-12)


def test_retarded_relation():
    # hand-worked: ((3 + 1i) - (1 - 1i)) / 2 = 1 + 1i; ((-2) - (4 + 2i)) / 2 = -3 - 1i
    np.testing.assert_array_equal(oracle.retarded(np.array([3 + 1j, -2]), np.array([1 - 1j, 4 + 2j])),
                                  np.array([1 + 1j, -3 - 1j]))
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 4, 2, 12, 12)) + 1j * rng.standard_normal((3, 4, 2, 12, 12))
    assert np.all(oracle.retarded(x, x) == 0)
    np.testing.assert_array_equal(oracle.retarded(x, -x), x)
