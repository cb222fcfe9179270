"""Communication-avoiding partition of the self-energy over processes (Section 3,
"Communication Avoidance") -- host logic for running the path on several GPUs.

The output points (kz, E, a) are independent.  The paper tiles the energies into T_E
ranges and the atoms into T_A ranges, P = T_E * T_A processes, each process owning one
(E-tile x atom-tile) shard and every kz.  A shard needs, for all kz:
  * G at the energies of its tile and up to omega_max below them (the halo of the
    one-sided E - omega access), for its atoms' neighbours (the atom halo: the paper
    approximates it by the tile plus N_B atoms, here it is taken exactly from the
    neighbour list);
  * Dt and dH of its own atoms.
Between the Green's-function phase (which owns whole (kz, E) rows of G) and the
self-energy phase, G moves once, by an all-to-all with per-destination counts
(alltoallv), and Sigma moves back the same way.  Per process the paper models the bytes
of G and Sigma as 64 Nkz (NE/T_E + 2 Nw)(NA/T_A + NB) Norb^2 and of D and Pi as
64 Nqz Nw (NA/T_A + NB) NB N3D^2 (double complex, both signs), against OMEN's
64 (Nkz NE / P) Nqz Nw NA Norb^2 and 64 Nqz Nw NA NB N3D^2; the tile sizes come from an
exhaustive search over the feasible (T_E, T_A).

Nothing here touches a GPU: the functions return index ranges, byte counts and plans
that a multi-GPU driver (one process per GPU, NCCL alltoallv) would execute.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Tuple

import numpy as np

NORB = 12
N3D = 3


# --- the paper's volume model ---------------------------------------------------------------

def volume_dace(nkz: int, nqz: int, ne: int, nw: int, na: int, nb: int, t_e: int, t_a: int,
                norb: int = NORB) -> float:
    """Bytes each process contributes to the all-to-all exchanges of the tiled scheme."""
    g = 64.0 * nkz * (ne / t_e + 2 * nw) * (na / t_a + nb) * norb * norb
    d = 64.0 * nqz * nw * (na / t_a + nb) * nb * N3D * N3D
    return g + d


def volume_omen(nkz: int, nqz: int, ne: int, nw: int, na: int, nb: int, p: int, norb: int = NORB) -> float:
    """Bytes each process receives / exchanges in OMEN's original distribution."""
    g = 64.0 * (nkz * ne / p) * nqz * nw * na * norb * norb
    d = 64.0 * nqz * nw * na * nb * N3D * N3D
    return g + d


def best_tiling(nkz: int, nqz: int, ne: int, nw: int, na: int, nb: int, p: int) -> Tuple[int, int, float]:
    """Exhaustive search over the feasible tilings T_E * T_A = P (T_E <= NE, T_A <= NA) for
    the smallest modelled volume per process; returns (T_E, T_A, bytes)."""
    best = None
    for t_e in range(1, p + 1):
        if p % t_e or t_e > ne or p // t_e > na:
            continue
        v = volume_dace(nkz, nqz, ne, nw, na, nb, t_e, p // t_e)
        if best is None or v < best[2]:
            best = (t_e, p // t_e, v)
    if best is None:
        raise ValueError(f"no feasible tiling of {p} processes over NE={ne}, NA={na}")
    return best


# --- shards and their halos ------------------------------------------------------------------

def split_range(n: int, parts: int, i: int) -> Tuple[int, int]:
    """Part i of [0, n) cut into `parts` nearly equal ranges (the first n % parts one longer)."""
    q, r = divmod(n, parts)
    lo = i * q + min(i, r)
    return lo, lo + q + (1 if i < r else 0)


@dataclasses.dataclass(frozen=True)
class Shard:
    index: int
    e0: int
    e1: int          # energies [e0, e1) of the output
    a0: int
    a1: int          # atoms [a0, a1) of the output
    e_lo: int        # first energy of G needed: max(0, e0 - omega_max)
    atoms: Tuple[int, ...]  # atoms of G needed: own atoms first, then the halo (ascending)


def make_shards(ne: int, na: int, nw: int, omega_first: int, neigh: np.ndarray, t_e: int, t_a: int) -> List[Shard]:
    """The T_E * T_A shards, energy tile major, with their exact halos."""
    omega_max = omega_first + nw - 1
    out = []
    for te in range(t_e):
        e0, e1 = split_range(ne, t_e, te)
        for ta in range(t_a):
            a0, a1 = split_range(na, t_a, ta)
            own = list(range(a0, a1))
            nbrs = set(int(f) for f in neigh[a0:a1].ravel() if f >= 0) - set(own)
            out.append(Shard(len(out), e0, e1, a0, a1, max(0, e0 - omega_max), tuple(own + sorted(nbrs))))
    return out


def local_problem(sh: Shard, G: np.ndarray, Dt: np.ndarray, dH: np.ndarray, neigh: np.ndarray) -> Dict[str, np.ndarray]:
    """The shard's inputs as a self-contained instance: G over energies [e_lo, e1) and the
    shard's atoms (own atoms at local indices 0 .. a1 - a0 - 1), the neighbour list
    re-indexed to local atoms (halo rows empty), Dt and dH of the own atoms (zero for the
    halo).  The self-energy of local energies e0 - e_lo .. e1 - e_lo - 1 and local atoms
    0 .. a1 - a0 - 1 is that shard's output: every term it needs lies inside the halo."""
    atoms = np.asarray(sh.atoms, dtype=np.int64)
    n_own = sh.a1 - sh.a0
    local_of = {int(a): i for i, a in enumerate(atoms)}
    lneigh = np.full((len(atoms), neigh.shape[1]), -1, dtype=np.int32)
    for i in range(n_own):
        for s, f in enumerate(neigh[sh.a0 + i]):
            lneigh[i, s] = local_of[int(f)] if f >= 0 else -1
    lG = np.ascontiguousarray(G[:, sh.e_lo:sh.e1][:, :, atoms])
    lDt = np.zeros(Dt.shape[:2] + (len(atoms),) + Dt.shape[3:], dtype=Dt.dtype)
    lDt[:, :, :n_own] = Dt[:, :, sh.a0:sh.a1]
    ldH = np.zeros((len(atoms),) + dH.shape[1:], dtype=dH.dtype)
    ldH[:n_own] = dH[sh.a0:sh.a1]
    return {"G": lG, "Dt": lDt, "dH": ldH, "neigh": lneigh}


# --- the exchange between the Green's-function layout and the shard layout ------------------

def gf_owner(nkz: int, ne: int, p: int) -> np.ndarray:
    """Owner process of each (kz, E) row in the Green's-function phase: the Nkz * NE
    independent (kz, E) problems dealt out in contiguous blocks, as the GF solver produces
    them.  Returns an int array [nkz, ne]."""
    flat = np.empty(nkz * ne, dtype=np.int64)
    for r in range(p):
        lo, hi = split_range(nkz * ne, p, r)
        flat[lo:hi] = r
    return flat.reshape(nkz, ne)


def exchange_plan(shards: List[Shard], owner: np.ndarray, shard_rank: List[int]) -> Dict[Tuple[int, int], List[Tuple[int, int, int, Tuple[int, ...]]]]:
    """What each process sends to each other one: {(src, dst): [(kz, E, shard index, atoms)]},
    in a fixed order (shard, kz, E) that the receiver reproduces.  `shard_rank[s]` is the
    process that evaluates shard s."""
    plan: Dict[Tuple[int, int], list] = {}
    nkz = owner.shape[0]
    for sh in shards:
        dst = shard_rank[sh.index]
        for k in range(nkz):
            for e in range(sh.e_lo, sh.e1):
                plan.setdefault((int(owner[k, e]), dst), []).append((k, e, sh.index, sh.atoms))
    return plan


def exchange_bytes(plan, elem_bytes: int = 16, norb: int = NORB) -> Dict[int, int]:
    """Bytes of G each process receives from others (one sign), per destination."""
    out: Dict[int, int] = {}
    for (src, dst), items in plan.items():
        if src == dst:
            continue
        out[dst] = out.get(dst, 0) + sum(len(atoms) for _, _, _, atoms in items) * norb * norb * elem_bytes
    return out
