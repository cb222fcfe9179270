"""Mixed-precision tensor-core kernel vs the CPU FP64 oracle, through the C ABI.

Tolerance: relative Frobenius error <= 2e-5 per sign (the mixed path's stated bound).
Cases span several tiles with a ragged last tile, every supported Nkz, qz wrap with
Nqz != Nkz, omega offsets, energies below the grid, empty / duplicate / self slots,
complex64 storage, and the full medium and precision workloads on sampled outputs.
"""
import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs
from tests.gpu_helpers import max_block_rel, rel_fro, run

pytestmark = pytest.mark.gpu
TOL = 2e-5


def oracle_full(inst, sign, omega_first=1):
    return oracle.sigma_atoms(inst["G_" + sign], inst["D_" + sign], inst["dH"], inst["neigh"],
                              omega_first=omega_first)


def test_tiny_config_both_signs():
    inst = inputs.make_instance(inputs.TINY, 0)
    out = run(inst, "mixed")
    for s in ("gt", "lt"):
        ref = oracle_full(inst, s)
        assert rel_fro(out[s], ref) <= TOL
        assert max_block_rel(out[s], ref) <= 1e-3
        # the anti-Hermiticity invariant survives the mixed arithmetic to its precision
        assert rel_fro(out[s], -np.conj(np.swapaxes(out[s], -1, -2))) <= 2 * TOL


@pytest.mark.parametrize("nkz", [1, 2, 3, 4, 5])
def test_every_supported_nkz(nkz):
    # NE = 3 tiles + a ragged tail for every tile height
    geo = inputs.Geometry(nkz=nkz, nqz=nkz, ne=3 * (128 // (3 * nkz)) + 5, nw=6, na=6, nb=4)
    inst = inputs.make_instance(geo, 30 + nkz)
    out = run(inst, "mixed")
    for s in ("gt", "lt"):
        assert rel_fro(out[s], oracle_full(inst, s)) <= TOL


@pytest.mark.parametrize("case", [
    dict(nkz=3, nqz=5, ne=40, nw=5, na=7, nb=3, omega_first=1),   # qz folds onto kz
    dict(nkz=4, nqz=2, ne=23, nw=6, na=5, nb=2, omega_first=0),   # omega_first = 0
    dict(nkz=2, nqz=2, ne=5, nw=9, na=6, nb=2, omega_first=2),    # most E - omega below the grid
    dict(nkz=1, nqz=1, ne=70, nw=16, na=1, nb=4, omega_first=1),  # one atom, self slots
    dict(nkz=5, nqz=5, ne=17, nw=32, na=3, nb=4, omega_first=1),  # Nw = 32 with a short grid
    dict(nkz=5, nqz=5, ne=21, nw=50, na=2, nb=2, omega_first=1),  # largest Nw of the warp-specialised form
    dict(nkz=5, nqz=5, ne=21, nw=56, na=2, nb=2, omega_first=1),  # past it: the single-role form takes over
    dict(nkz=3, nqz=3, ne=37, nw=17, na=5, nb=3, omega_first=-8),  # two-sided grid, single-role form
    dict(nkz=5, nqz=5, ne=30, nw=33, na=4, nb=3, omega_first=-16), # two-sided grid, warp-specialised form
    dict(nkz=5, nqz=5, ne=12, nw=9, na=3, nb=2, omega_first=-12),  # all frequencies negative
])
def test_edge_geometries(case):
    of = case.pop("omega_first")
    geo = inputs.Geometry(norb=12, omega_first=of, **case)
    rng = np.random.default_rng(9)
    neigh = rng.integers(0, geo.na, size=(geo.na, geo.nb)).astype(np.int32)
    inst = inputs.make_instance(geo, 41, neigh=neigh, hermitian_pairs=False)
    out = run(inst, "mixed", omega_first=of)
    for s in ("gt", "lt"):
        assert rel_fro(out[s], oracle_full(inst, s, of)) <= TOL


def test_empty_duplicate_slots_single_sign_and_isolated_atom():
    geo = inputs.Geometry(nkz=3, nqz=3, ne=30, nw=4, na=9, nb=5)
    neigh = inputs.chain_neighbours(9, (-2, -1, 1, 2, 1))
    neigh[3, 1] = -1
    neigh[7, :] = -1
    inst = inputs.make_instance(geo, 23, neigh=neigh, hermitian_pairs=False)
    out = run(inst, "mixed", signs=("gt",))
    assert rel_fro(out["gt"], oracle_full(inst, "gt")) <= TOL
    assert np.all(out["gt"][:, :, 7] == 0)


def test_complex64_batched_shape():
    """One instance shaped like the batched workload: Nkz=Nqz=3, Nw=16, per-atom
    neighbour counts 3..8 within +-8 sites, complex64 storage."""
    rng = np.random.default_rng(3)
    na, ne = 150, 77
    neigh = inputs.random_neighbours(rng, na, nb_max=8)
    geo = inputs.Geometry(nkz=3, nqz=3, ne=ne, nw=16, na=na, nb=8)
    inst = inputs.make_instance(geo, 5, dtype=np.complex64, neigh=neigh, hermitian_pairs=False)
    out = run(inst, "mixed")
    for s in ("gt", "lt"):
        assert rel_fro(out[s], oracle_full(inst, s)) <= TOL


def test_mixed_matches_fp64_kernel_on_tiny():
    inst = inputs.make_instance(inputs.TINY, 7)
    a = run(inst, "mixed")
    b = run(inst, "fp64")
    for s in ("gt", "lt"):
        assert rel_fro(a[s], b[s]) <= TOL


def sampled_points(geo, n, seed):
    rng = np.random.default_rng(seed)
    pts = [(0, 0, 0), (geo.nkz - 1, geo.ne - 1, geo.na - 1), (1, 1, 3), (2, geo.nw, 100 % geo.na),
           (geo.nkz - 1, geo.nw + 1, geo.na // 2)]
    pts += [tuple(int(x) for x in (rng.integers(geo.nkz), rng.integers(geo.ne), rng.integers(geo.na)))
            for _ in range(n)]
    return pts


def test_medium_config_across_the_atom_axis():
    """Full medium workload (the benchmark's launch: the warp-specialised form with units of
    16 energy tiles) against the oracle element by element on five 16-atom ranges spread
    over the atom axis (every (kz, E) of 80 atoms, both signs), plus sampled single blocks
    and whole-tensor invariants."""
    geo = inputs.MEDIUM
    inst = inputs.make_instance(geo, 1)
    out = run(inst, "mixed")
    ranges = [(0, 16), (120, 136), (248, 264), (376, 392), (496, 512)]
    pts = sampled_points(geo, 12, 0)
    for s in ("gt", "lt"):
        for a0, a1 in ranges:
            ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], a0, a1)
            assert rel_fro(out[s][:, :, a0:a1], ref) <= TOL, (s, a0)
            assert max_block_rel(out[s][:, :, a0:a1], ref) <= 1e-3
        refp = oracle.sigma_points(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], pts)
        got = np.stack([out[s][k, e, a] for k, e, a in pts])
        assert rel_fro(got, refp) <= TOL
        assert np.all(out[s][:, 0] == 0)
        assert np.all(np.isfinite(out[s]))
        assert rel_fro(out[s], -np.conj(np.swapaxes(out[s], -1, -2))) <= 2 * TOL


def test_precision_config_128_atom_slice_both_signs():
    """Precision workload (Na = 2048, G about 6 GB per sign in complex128, seed 2): the error
    against the oracle on the Na = 128 atom slice, element by element, for both signs."""
    geo = inputs.PRECISION
    inst = inputs.make_instance(geo, 2)
    out = run(inst, "mixed")
    for s in ("gt", "lt"):
        ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], 0, 128)
        assert rel_fro(out[s][:, :, 0:128], ref) <= TOL, s
        pts = sampled_points(geo, 8, 1)
        refp = oracle.sigma_points(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], pts)
        got = np.stack([out[s][k, e, a] for k, e, a in pts])
        assert rel_fro(got, refp) <= TOL


@pytest.mark.parametrize("case", [
    dict(ne=45, nw=32, na=9, nb=4, chain=True),    # ragged last tile, four slots per atom
    dict(ne=20, nw=12, na=7, nb=6, chain=False),   # random slots incl. duplicates and self
])
def test_warp_specialised_form_complex64(case):
    """Nkz = 5 with complex64 storage runs the warp-specialised kernel with float2 output:
    the first slot's store and every later slot's FP32 reduction in place."""
    geo = inputs.Geometry(nkz=5, nqz=5, ne=case["ne"], nw=case["nw"], na=case["na"], nb=case["nb"])
    if case["chain"]:
        inst = inputs.make_instance(geo, 71, dtype=np.complex64)
    else:
        rng = np.random.default_rng(72)
        neigh = rng.integers(0, geo.na, size=(geo.na, geo.nb)).astype(np.int32)
        neigh[0, 1] = -1
        inst = inputs.make_instance(geo, 73, dtype=np.complex64, neigh=neigh, hermitian_pairs=False)
    plans = []
    out = run(inst, "mixed", plan_out=plans)
    assert plans[0].info().workspace_bytes > 1024  # the warp-specialised form's workspace
    plans[0].close()
    for s in ("gt", "lt"):
        assert rel_fro(out[s], oracle_full(inst, s)) <= TOL

