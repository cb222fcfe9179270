"""The phonon self-energy Pi (Eq. 5 off-diagonal blocks, Eq. 4 diagonal block) on the GPU,
through the C ABI, against the CPU FP64 oracle element by element.

Tolerances: relative Frobenius error <= 1e-11 per sign for complex128 (FP64 throughout, only
the summation order differs), <= 1e-6 for complex64 storage (the result is rounded once to
FP32)."""
import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, to_device

pytestmark = pytest.mark.gpu


def run_pi(inst, nqz, nw, omega_first=1, signs=("gt", "lt")):
    import torch
    dev = to_device(inst)
    nkz, ne, na = inst["G_gt"].shape[:3]
    nb = inst["neigh"].shape[1]
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=nkz, nqz=nqz, ne=ne, nw=nw, omega_first=omega_first, mode="fp64")
    out = {s: (torch.full((nqz, nw, na, nb + 1, 3, 3), float("nan"), dtype=dev["G_gt"].dtype, device="cuda")
               if s in signs else None) for s in ("gt", "lt")}
    plan.pi(dev["G_gt"], dev["G_lt"], out["gt"], out["lt"])
    torch.cuda.synchronize()
    plan.close()
    return {s: out[s].cpu().numpy() for s in signs}


def ref_pi(inst, sign, nqz, nw, omega_first=1):
    other = "lt" if sign == "gt" else "gt"
    return oracle.pi(inst["G_" + sign], inst["G_" + other], inst["dH"], inst["neigh"], nqz, nw, omega_first)


@pytest.mark.parametrize("case", [
    dict(nkz=3, nqz=3, ne=20, nw=4, na=9, nb=4, of=1, dtype=np.complex128, chain=True),
    dict(nkz=5, nqz=5, ne=40, nw=32, na=6, nb=4, of=1, dtype=np.complex128, chain=True),   # medium's Nw
    dict(nkz=4, nqz=2, ne=13, nw=6, na=7, nb=3, of=0, dtype=np.complex128, chain=False),  # Nqz != Nkz, omega_first 0
    dict(nkz=2, nqz=3, ne=9, nw=11, na=5, nb=2, of=2, dtype=np.complex128, chain=False),  # Nqz > Nkz, most E + w off the grid
    dict(nkz=3, nqz=3, ne=25, nw=16, na=8, nb=8, of=1, dtype=np.complex64, chain=False),  # batched-like, complex64
    dict(nkz=1, nqz=1, ne=30, nw=1, na=4, nb=4, of=1, dtype=np.complex128, chain=False),  # Nw = 1
    dict(nkz=3, nqz=3, ne=18, nw=9, na=5, nb=3, of=-4, dtype=np.complex128, chain=False),  # two-sided grid
])
def test_pi_matches_oracle(case):
    geo = inputs.Geometry(nkz=case["nkz"], nqz=case["nqz"], ne=case["ne"], nw=case["nw"], na=case["na"],
                          nb=case["nb"], omega_first=case["of"])
    if case["chain"]:
        inst = inputs.make_instance(geo, 11, dtype=case["dtype"])
    else:
        rng = np.random.default_rng(12)
        neigh = rng.integers(-1, geo.na, size=(geo.na, geo.nb)).astype(np.int32)  # empty, duplicate, self slots
        inst = inputs.make_instance(geo, 13, dtype=case["dtype"], neigh=neigh, hermitian_pairs=False)
    tol = 1e-11 if case["dtype"] == np.complex128 else 1e-6
    got = run_pi(inst, geo.nqz, geo.nw, geo.omega_first)
    for s in ("gt", "lt"):
        ref = ref_pi(inst, s, geo.nqz, geo.nw, geo.omega_first)
        assert rel_fro(got[s], ref) <= tol, s
        # Hermitian in (i, j): both G anti-Hermitian
        assert rel_fro(got[s], np.conj(np.swapaxes(got[s], -1, -2))) <= 10 * tol


def test_pi_single_sign_more_atoms_than_sms():
    """One sign only, and more CTAs (one per atom) than the GPU has SMs."""
    geo = inputs.Geometry(nkz=3, nqz=3, ne=12, nw=4, na=160, nb=4)
    inst = inputs.make_instance(geo, 14)
    got = run_pi(inst, 3, 4, signs=("lt",))
    assert rel_fro(got["lt"], ref_pi(inst, "lt", 3, 4)) <= 1e-11
