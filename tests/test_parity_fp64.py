"""FP64 direct kernel vs the CPU FP64 oracle, element by element, through the C ABI.

Tolerance: relative Frobenius error <= 1e-11 per sign for complex128 storage (the FP64
path's stated bound); complex64 storage rounds the stored output, so 1e-6 there.
"""
import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs
from tests.gpu_helpers import max_block_rel, rel_fro, run

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


def oracle_full(inst, sign, omega_first=1):
    return oracle.sigma_atoms(inst["G_" + sign], inst["D_" + sign], inst["dH"], inst["neigh"],
                              omega_first=omega_first)


def test_tiny_config_both_signs():
    inst = inputs.make_instance(inputs.TINY, 0)
    out = run(inst, "fp64")
    for s in ("gt", "lt"):
        ref = oracle_full(inst, s)
        assert rel_fro(out[s], ref) <= TOL64
        assert max_block_rel(out[s], ref) <= 1e-10
        # anti-Hermitian, as the oracle's invariant promises for these inputs
        assert rel_fro(out[s], -np.conj(np.swapaxes(out[s], -1, -2))) <= 1e-12


@pytest.mark.parametrize("case", [
    dict(nkz=3, nqz=5, ne=20, nw=3, na=7, nb=3, omega_first=1),   # nqz > nkz
    dict(nkz=4, nqz=2, ne=9, nw=6, na=5, nb=2, omega_first=0),    # omega_first = 0
    dict(nkz=2, nqz=2, ne=3, nw=8, na=6, nb=2, omega_first=2),    # most E - omega below the grid
    dict(nkz=1, nqz=1, ne=33, nw=5, na=1, nb=4, omega_first=1),   # one atom, one k
    dict(nkz=3, nqz=3, ne=21, nw=9, na=6, nb=3, omega_first=-4),  # two-sided grid: E -+ omega
])
def test_edge_geometries(case):
    of = case.pop("omega_first")
    geo = inputs.Geometry(norb=12, omega_first=of, **case)
    rng = np.random.default_rng(5)
    neigh = rng.integers(0, geo.na, size=(geo.na, geo.nb)).astype(np.int32)
    inst = inputs.make_instance(geo, 17, neigh=neigh, hermitian_pairs=False)
    out = run(inst, "fp64", omega_first=of)
    for s in ("gt", "lt"):
        assert rel_fro(out[s], oracle_full(inst, s, of)) <= TOL64


def test_empty_and_duplicate_slots_and_single_sign():
    geo = inputs.Geometry(nkz=3, nqz=3, ne=16, nw=4, na=9, nb=5)
    neigh = inputs.chain_neighbours(9, (-2, -1, 1, 2, 1))  # slot 4 duplicates slot 2
    neigh[3, 1] = -1
    neigh[7, :] = -1                                       # an atom with no neighbours
    inst = inputs.make_instance(geo, 23, neigh=neigh, hermitian_pairs=False)
    out = run(inst, "fp64", signs=("lt",))
    ref = oracle_full(inst, "lt")
    assert rel_fro(out["lt"], ref) <= TOL64
    assert np.all(out["lt"][:, :, 7] == 0)


def test_complex64_storage():
    inst = inputs.make_instance(inputs.TINY, 4, dtype=np.complex64)
    out = run(inst, "fp64")
    for s in ("gt", "lt"):
        assert rel_fro(out[s], oracle_full(inst, s)) <= 1e-6


def test_medium_config_sampled_points():
    """Full medium size (Nkz=Nqz=5, NE=256, Nw=32, Na=512, Nb=4, seed 1), checked on
    sampled output blocks that the oracle evaluates one by one."""
    inst = inputs.make_instance(inputs.MEDIUM, 1)
    out = run(inst, "fp64")
    g = inputs.MEDIUM
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (g.nkz - 1, g.ne - 1, g.na - 1), (2, 1, 5), (1, 31, 200), (3, 32, 511),
           (4, 33, 17)] + [tuple(int(x) for x in (rng.integers(g.nkz), rng.integers(g.ne), rng.integers(g.na)))
                           for _ in range(10)]
    for s in ("gt", "lt"):
        ref = oracle.sigma_points(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], pts)
        got = np.stack([out[s][k, e, a] for k, e, a in pts])
        assert rel_fro(got, ref) <= TOL64
        assert np.all(out[s][:, 0] == 0)
