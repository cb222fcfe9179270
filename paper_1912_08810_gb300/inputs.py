"""Seeded synthetic inputs for the electron scattering self-energy (Eq. 3).

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Both the CUDA path and the CPU oracle consume the bytes it
produces, so parity never depends on the generator.

Layout (row-major, complex values with real/imaginary parts interleaved), as the
tensors are described in Section 3 ("Dataflow Optimizations", the 5-D G and
6-D D tensors of Section 2):

  G^>, G^<   [nkz][ne][na][norb][norb]      electron Green's functions, diagonal blocks
  Dt^>, Dt^< [nqz][nw][na][nb][3][3]        pre-combined phonon term D_ba - D_bb - D_aa + D_ab
  dH         [na][nb][3][norb][norb]        gradient blocks  grad_i H_{a, neigh[a,b]}
  neigh      [na][nb] int32                 neighbour atom of slot b, -1 = empty slot

Value recipe (the workloads of Table 1 have no published inputs, so these stand in):
  * G blocks are A - A^dagger with Re A, Im A ~ N(0, 1) independently (anti-Hermitian,
    like physical lesser/greater Green's functions);
  * dH blocks are complex normal; on the periodic chain the reverse bond block is the
    conjugate transpose, dH[b, slot(a)] = dH[a, slot(b)]^dagger;
  * Dt blocks are B + B^dagger (3x3 Hermitian) with B complex normal.
Draw order from ``numpy.random.default_rng(seed)``: G^>, G^<, dH, Dt^>, Dt^<; each
complex array is drawn as one float64 normal array of shape (..., 2) in C order.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

N3D = 3


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Sizes of one SSE instance (symbols of Table 1)."""
    nkz: int
    nqz: int
    ne: int
    nw: int
    na: int
    nb: int
    norb: int = 12
    omega_first: int = 1  # the phonon frequency w is (w + omega_first) energy-grid steps

    def points(self) -> int:
        """Output blocks (kz, E, a) per sign."""
        return self.nkz * self.ne * self.na


# Named workloads.  Shapes follow Table 1 ranges scaled to one GPU.
TINY = Geometry(nkz=3, nqz=3, ne=48, nw=4, na=16, nb=4)
MEDIUM = Geometry(nkz=5, nqz=5, ne=256, nw=32, na=512, nb=4)
PRECISION = Geometry(nkz=5, nqz=5, ne=256, nw=32, na=2048, nb=4)

CHAIN_OFFSETS = (-2, -1, 1, 2)


def chain_neighbours(na: int, offsets=CHAIN_OFFSETS) -> np.ndarray:
    """Periodic-chain neighbour list: slot s of atom a is (a + offsets[s]) mod na."""
    a = np.arange(na, dtype=np.int64)[:, None]
    return ((a + np.asarray(offsets, dtype=np.int64)[None, :]) % na).astype(np.int32)


def _complex_normal(rng: np.random.Generator, shape, chunk_rows: int = 1 << 16) -> np.ndarray:
    """Complex normal array (Re, Im ~ N(0,1)) drawn as float64 pairs in C order.

    Drawn in chunks along the leading axis so peak host memory stays near the output
    size; the chunking does not change the stream of values.
    """
    shape = tuple(int(s) for s in shape)
    out = np.empty(shape, dtype=np.complex128)
    flat = out.reshape(shape[0], -1) if len(shape) > 1 else out.reshape(-1, 1)
    rows = flat.shape[0]
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        x = rng.standard_normal((r1 - r0, flat.shape[1], 2))
        flat[r0:r1] = x[..., 0] + 1j * x[..., 1]
    return out


def _anti_hermitian_blocks(rng, lead_shape, norb) -> np.ndarray:
    a = _complex_normal(rng, tuple(lead_shape) + (norb, norb))
    a -= np.conj(np.swapaxes(a, -1, -2)).copy()
    return a


def _hermitian_3x3(rng, lead_shape) -> np.ndarray:
    b = _complex_normal(rng, tuple(lead_shape) + (N3D, N3D))
    return np.ascontiguousarray(b + np.conj(np.swapaxes(b, -1, -2)))


def make_instance(geo: Geometry, seed: int, *, dtype=np.complex128,
                  neigh: Optional[np.ndarray] = None,
                  hermitian_pairs: Optional[bool] = None) -> Dict[str, np.ndarray]:
    """One seeded instance: dict with G_gt, G_lt, D_gt, D_lt, dH, neigh.

    ``neigh`` defaults to the periodic chain with offsets (-2, -1, +1, +2) when
    ``geo.nb == 4``.  ``hermitian_pairs`` (default: True for the chain) makes the
    reverse bond block the conjugate transpose of the forward one.
    """
    rng = np.random.default_rng(seed)
    if neigh is None:
        if geo.nb != len(CHAIN_OFFSETS):
            raise ValueError("default chain neighbours need nb == 4")
        neigh = chain_neighbours(geo.na)
        if hermitian_pairs is None:
            hermitian_pairs = True
    neigh = np.ascontiguousarray(neigh, dtype=np.int32)
    assert neigh.shape == (geo.na, geo.nb)
    lead_g = (geo.nkz, geo.ne, geo.na)
    g_gt = _anti_hermitian_blocks(rng, lead_g, geo.norb)
    g_lt = _anti_hermitian_blocks(rng, lead_g, geo.norb)
    dh = _complex_normal(rng, (geo.na, geo.nb, N3D, geo.norb, geo.norb))
    if hermitian_pairs:
        _make_reverse_bonds_hermitian(dh, neigh)
    lead_d = (geo.nqz, geo.nw, geo.na, geo.nb)
    d_gt = _hermitian_3x3(rng, lead_d)
    d_lt = _hermitian_3x3(rng, lead_d)
    out = dict(G_gt=g_gt, G_lt=g_lt, D_gt=d_gt, D_lt=d_lt, dH=dh, neigh=neigh)
    for k in ("G_gt", "G_lt", "D_gt", "D_lt", "dH"):
        out[k] = np.ascontiguousarray(out[k], dtype=dtype)
    return out


def _make_reverse_bonds_hermitian(dh: np.ndarray, neigh: np.ndarray) -> None:
    """For each bond a -> b that also appears as b -> a, set dH[b, slot of a] = dH[a, slot of b]^dagger.

    The forward block of each unordered pair is the one stored at the lower
    (atom, slot) position in C order; only bonds present in both lists are paired.
    """
    na, nb = neigh.shape
    done = set()
    for a in range(na):
        for s in range(nb):
            b = int(neigh[a, s])
            if b < 0 or (a, s) in done:
                continue
            rev = [t for t in range(nb) if int(neigh[b, t]) == a and (b, t) not in done]
            if not rev or (b == a):
                continue
            t = rev[0]
            dh[b, t] = np.conj(np.swapaxes(dh[a, s], -1, -2))
            done.add((a, s))
            done.add((b, t))


def random_neighbours(rng: np.random.Generator, na: int, nb_max: int = 8,
                      nb_lo: int = 3, nb_hi: int = 8, reach: int = 8) -> np.ndarray:
    """Random neighbour lists: per atom nb ~ U{nb_lo..nb_hi} distinct atoms within
    +-reach sites (mod na, never the atom itself); unused slots are -1."""
    neigh = np.full((na, nb_max), -1, dtype=np.int32)
    offs = np.array([o for o in range(-reach, reach + 1) if o != 0], dtype=np.int64)
    for a in range(na):
        n = int(rng.integers(nb_lo, nb_hi + 1))
        cand = np.unique((a + offs) % na)
        cand = cand[cand != a]
        n = min(n, cand.size)
        pick = rng.choice(cand, size=n, replace=False)
        neigh[a, :n] = pick.astype(np.int32)
    return neigh


@dataclasses.dataclass
class BatchedSpec:
    """Batched workload: many independent instances of uneven size (Nkz=Nqz=3, Nw=16)."""
    n_instances: int = 64
    na_range: tuple = (64, 1024)
    ne_range: tuple = (64, 512)
    nkz: int = 3
    nw: int = 16
    nb_max: int = 8
    nb_range: tuple = (3, 8)
    reach: int = 8


def batched_geometries(spec: BatchedSpec, seed: int) -> List[Geometry]:
    """Sizes of each instance of the batched workload (drawn before any values)."""
    rng = np.random.default_rng(seed)
    geos = []
    for _ in range(spec.n_instances):
        na = int(rng.integers(spec.na_range[0], spec.na_range[1] + 1))
        ne = int(rng.integers(spec.ne_range[0], spec.ne_range[1] + 1))
        geos.append(Geometry(nkz=spec.nkz, nqz=spec.nkz, ne=ne, nw=spec.nw, na=na,
                             nb=spec.nb_max))
    return geos


def make_batched(spec: BatchedSpec, seed: int, *, dtype=np.complex64,
                 which: Optional[List[int]] = None) -> List[Dict[str, np.ndarray]]:
    """Instances of the batched workload; instance i uses seed (seed, i) so any subset
    can be generated alone and still match the full set."""
    geos = batched_geometries(spec, seed)
    idx = range(len(geos)) if which is None else which
    out = []
    for i in idx:
        g = geos[i]
        nrng = np.random.default_rng([seed, i, 1])
        neigh = random_neighbours(nrng, g.na, spec.nb_max, spec.nb_range[0],
                                  spec.nb_range[1], spec.reach)
        inst = make_instance(g, seed=int(np.random.SeedSequence([seed, i, 2]).generate_state(1)[0]),
                             dtype=dtype, neigh=neigh, hermitian_pairs=False)
        inst["geometry"] = g
        out.append(inst)
    return out


def make_instance_torch(geo: Geometry, seed: int, *, device="cuda", dtype=None,
                        neigh: Optional[np.ndarray] = None, hermitian_pairs: Optional[bool] = None):
    """Same recipe as make_instance, drawn on the device with torch's counter-based
    generator (for workloads too large to draw on the host).  Values differ from the
    numpy draw of the same seed; tests that compare with the CPU oracle copy these
    tensors to the host, so both sides still consume the same bytes.  Returns a dict of
    torch tensors (complex64 by default)."""
    import torch
    dtype = dtype or torch.complex64
    real = torch.float32 if dtype == torch.complex64 else torch.float64
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    if neigh is None:
        if geo.nb != len(CHAIN_OFFSETS):
            raise ValueError("default chain neighbours need nb == 4")
        neigh = chain_neighbours(geo.na)
        if hermitian_pairs is None:
            hermitian_pairs = True
    neigh_np = np.ascontiguousarray(neigh, dtype=np.int32)

    def cnormal(shape):
        x = torch.randn(tuple(shape) + (2,), generator=gen, device=device, dtype=real)
        return torch.view_as_complex(x)

    def anti_herm(shape):
        a = cnormal(shape)
        return (a - a.transpose(-1, -2).conj()).contiguous()

    def herm(shape):
        b = cnormal(shape)
        return (b + b.transpose(-1, -2).conj()).contiguous()

    lead_g = (geo.nkz, geo.ne, geo.na, geo.norb, geo.norb)
    out = {"G_gt": anti_herm(lead_g), "G_lt": anti_herm(lead_g)}
    dh = cnormal((geo.na, geo.nb, N3D, geo.norb, geo.norb))
    if hermitian_pairs:
        dh_np = dh.cpu().numpy()
        _make_reverse_bonds_hermitian(dh_np, neigh_np)
        dh = torch.from_numpy(dh_np).to(device)
    out["dH"] = dh.contiguous()
    lead_d = (geo.nqz, geo.nw, geo.na, geo.nb, N3D, N3D)
    out["D_gt"] = herm(lead_d)
    out["D_lt"] = herm(lead_d)
    out["neigh"] = torch.from_numpy(neigh_np).to(device)
    return out


def make_batched_torch(spec: BatchedSpec, seed: int, *, device="cuda", which: Optional[List[int]] = None):
    """The batched workload drawn on the device: instance i uses neighbour lists from
    numpy seed (seed, i, 1) (as make_batched) and values from torch seed (seed, i, 2)."""
    geos = batched_geometries(spec, seed)
    idx = range(len(geos)) if which is None else which
    out = []
    for i in idx:
        g = geos[i]
        nrng = np.random.default_rng([seed, i, 1])
        neigh = random_neighbours(nrng, g.na, spec.nb_max, spec.nb_range[0], spec.nb_range[1], spec.reach)
        vseed = int(np.random.SeedSequence([seed, i, 2]).generate_state(1)[0])
        inst = make_instance_torch(g, vseed, device=device, neigh=neigh, hermitian_pairs=False)
        inst["geometry"] = g
        out.append(inst)
    return out


def make_phonon_full(geo: Geometry, seed: int, neigh: np.ndarray, *, dtype=np.complex128) -> Dict[str, np.ndarray]:
    """Full phonon tensors D^>, D^< [nqz][nw][na][nb+1][3][3] (Section 2's shape: block nb of
    an atom is its diagonal block), complex normal, with the structure of a Hermitian
    matrix in (atom, direction): diagonal blocks B + B^dagger, and for each bond listed in
    both directions the reverse block the conjugate transpose of the forward one.  Draw
    order from default_rng(seed): D^> then D^<."""
    rng = np.random.default_rng(seed)
    neigh = np.ascontiguousarray(neigh, dtype=np.int32)
    na, nb = neigh.shape
    out = {}
    for name in ("D_gt_full", "D_lt_full"):
        d = _complex_normal(rng, (geo.nqz, geo.nw, na, nb + 1, N3D, N3D))
        d[:, :, :, nb] = d[:, :, :, nb] + np.conj(np.swapaxes(d[:, :, :, nb], -1, -2))
        done = set()
        for a in range(na):
            for s in range(nb):
                b = int(neigh[a, s])
                if b < 0 or (a, s) in done:
                    continue
                rev = [t for t in range(nb) if int(neigh[b, t]) == a and (b, t) not in done]
                if not rev or b == a:
                    continue
                d[:, :, b, rev[0]] = np.conj(np.swapaxes(d[:, :, a, s], -1, -2))
                done.add((a, s))
                done.add((b, rev[0]))
        out[name] = np.ascontiguousarray(d, dtype=dtype)
    return out
