"""Seeded input generators: structure the workloads promise (no method arithmetic here)."""
import numpy as np

from paper_1912_08810_gb300 import inputs


def test_tiny_structure_and_determinism():
    a = inputs.make_instance(inputs.TINY, 0)
    b = inputs.make_instance(inputs.TINY, 0)
    c = inputs.make_instance(inputs.TINY, 1)
    for k in ("G_gt", "G_lt", "D_gt", "D_lt", "dH", "neigh"):
        assert np.array_equal(a[k], b[k])
    assert not np.array_equal(a["G_gt"], c["G_gt"])
    g = inputs.TINY
    assert a["G_gt"].shape == (g.nkz, g.ne, g.na, 12, 12)
    assert a["D_gt"].shape == (g.nqz, g.nw, g.na, g.nb, 3, 3)
    assert a["dH"].shape == (g.na, g.nb, 3, 12, 12)
    for s in ("G_gt", "G_lt"):  # anti-Hermitian blocks
        G = a[s]
        assert np.array_equal(G, -np.conj(np.swapaxes(G, -1, -2)))
    for s in ("D_gt", "D_lt"):  # Hermitian 3x3 blocks
        D = a[s]
        assert np.array_equal(D, np.conj(np.swapaxes(D, -1, -2)))


def test_chain_neighbours_and_reverse_bonds():
    inst = inputs.make_instance(inputs.TINY, 0)
    neigh, dH = inst["neigh"], inst["dH"]
    na = neigh.shape[0]
    assert np.array_equal(neigh[5], [3, 4, 6, 7])
    assert np.array_equal(neigh[0], [na - 2, na - 1, 1, 2])
    for a in range(na):
        for s in range(4):
            b = neigh[a, s]
            t = list(neigh[b]).index(a)
            assert np.array_equal(dH[b, t], np.conj(np.swapaxes(dH[a, s], -1, -2)))


def test_random_neighbours_within_reach():
    rng = np.random.default_rng(3)
    neigh = inputs.random_neighbours(rng, 100, nb_max=8)
    for a in range(100):
        row = neigh[a]
        used = row[row >= 0]
        assert 3 <= used.size <= 8
        assert np.all(row[used.size:] == -1)
        assert len(set(used.tolist())) == used.size and a not in used
        d = np.minimum((used - a) % 100, (a - used) % 100)
        assert np.all(d <= 8)


def test_batched_subset_matches_full_draw():
    spec = inputs.BatchedSpec(n_instances=4, na_range=(16, 40), ne_range=(8, 20))
    full = inputs.make_batched(spec, 3)
    one = inputs.make_batched(spec, 3, which=[2])[0]
    assert full[2]["geometry"] == one["geometry"]
    for k in ("G_gt", "D_lt", "dH", "neigh"):
        assert np.array_equal(full[2][k], one[k])
    assert full[0]["G_gt"].dtype == np.complex64


def test_every_array_is_c_contiguous():
    for dt in (np.complex128, np.complex64):
        inst = inputs.make_instance(inputs.TINY, 2, dtype=dt)
        for k in ("G_gt", "G_lt", "D_gt", "D_lt", "dH", "neigh"):
            assert inst[k].flags.c_contiguous, k
