"""The steps on either side of Sigma on the GPU, through the C ABI, against the oracle:
the phonon pre-combination Dt = D_ba - D_bb - D_aa + D_ab (Eq. 3; Section 3 input list)
and Sigma^R = (Sigma^> - Sigma^<) / 2 (Section 2), alone and chained with the self-energy
(sse_execute_full).  Both steps are exact FP64 sums in a fixed order, so they are compared
bit for bit; the chained self-energy within the path's tolerance."""
import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, to_device

pytestmark = pytest.mark.gpu
TOL = {"mixed": 2e-5, "fp64": 1e-11}


def setup(geo, seed, dtype=np.complex128):
    import torch
    inst = inputs.make_instance(geo, seed, dtype=dtype)
    full = inputs.make_phonon_full(geo, seed + 100, inst["neigh"], dtype=dtype)
    dev = to_device(inst)
    for k in full:
        dev[k] = torch.from_numpy(full[k]).cuda()
    return inst, full, dev


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_dtilde_matches_oracle_exactly(dtype):
    import torch
    geo = inputs.Geometry(nkz=3, nqz=3, ne=8, nw=16, na=50, nb=4)
    inst, full, dev = setup(geo, 3, dtype)
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=3, nqz=3, ne=8, nw=16, mode="fp64")
    for s in ("gt", "lt"):
        Dt = torch.full_like(dev["D_gt"], float("nan"))
        plan.dtilde(dev[f"D_{s}_full"], Dt)
        torch.cuda.synchronize()
        ref = oracle.dtilde(full[f"D_{s}_full"], inst["neigh"]).astype(dtype)
        np.testing.assert_array_equal(Dt.cpu().numpy(), ref)
    plan.close()


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_retarded_matches_oracle_exactly(dtype):
    import torch
    geo = inputs.Geometry(nkz=3, nqz=3, ne=37, nw=4, na=11, nb=4)
    inst, _, dev = setup(geo, 4, dtype)
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=3, nqz=3, ne=37, nw=4, mode="fp64")
    S_r = torch.full_like(dev["G_gt"], float("nan"))
    plan.retarded(dev["G_gt"], dev["G_lt"], S_r)  # any two tensors of Sigma's shape
    torch.cuda.synchronize()
    ref = oracle.retarded(inst["G_gt"], inst["G_lt"]).astype(dtype)
    np.testing.assert_array_equal(S_r.cpu().numpy(), ref)
    plan.close()


@pytest.mark.parametrize("mode,geo,dtype", [
    ("mixed", inputs.Geometry(nkz=5, nqz=5, ne=45, nw=32, na=10, nb=4), np.complex128),  # warp-specialised
    ("mixed", inputs.Geometry(nkz=5, nqz=5, ne=21, nw=12, na=8, nb=4), np.complex64),
    ("mixed", inputs.Geometry(nkz=3, nqz=4, ne=50, nw=16, na=9, nb=4), np.complex64),    # single-role form
    ("fp64", inputs.Geometry(nkz=3, nqz=3, ne=30, nw=6, na=8, nb=4), np.complex128),
])
def test_execute_full_chain(mode, geo, dtype):
    """sse_execute_full from the full phonon tensors equals sse_dtilde + sse_execute bit for
    bit, and the oracle's chain (dtilde, Sigma, retarded) within the path's tolerance; the
    anti-Hermiticity invariant of Sigma holds through the pre-combination."""
    import torch
    inst, full, dev = setup(geo, 5, dtype)
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=geo.nkz, nqz=geo.nqz, ne=geo.ne, nw=geo.nw, mode=mode)
    S = {s: torch.full_like(dev["G_gt"], float("nan")) for s in ("gt", "lt", "r")}
    plan.execute_full(dev["G_gt"], dev["G_lt"], dev["D_gt_full"], dev["D_lt_full"], S["gt"], S["lt"], S["r"])
    Dt = {s: torch.empty_like(dev["D_gt"]) for s in ("gt", "lt")}
    for s in ("gt", "lt"):
        plan.dtilde(dev[f"D_{s}_full"], Dt[s])
    T = {s: torch.full_like(dev["G_gt"], float("nan")) for s in ("gt", "lt")}
    plan.execute(dev["G_gt"], dev["G_lt"], Dt["gt"], Dt["lt"], T["gt"], T["lt"])
    torch.cuda.synchronize()
    plan.status()
    for s in ("gt", "lt"):
        assert torch.equal(S[s], T[s])
    ref = {}
    for s in ("gt", "lt"):
        dt = oracle.dtilde(full[f"D_{s}_full"], inst["neigh"])
        ref[s] = oracle.sigma_atoms(inst["G_" + s], dt, inst["dH"], inst["neigh"])
        got = S[s].cpu().numpy()
        assert rel_fro(got, ref[s]) <= TOL[mode], s
        assert rel_fro(got, -np.conj(np.swapaxes(got, -1, -2))) <= 2 * TOL[mode]
    assert rel_fro(S["r"].cpu().numpy(), oracle.retarded(ref["gt"], ref["lt"])) <= TOL[mode]
    np.testing.assert_array_equal(S["r"].cpu().numpy(),
                                  oracle.retarded(S["gt"].cpu().numpy(), S["lt"].cpu().numpy()).astype(dtype))
    plan.close()


def test_bond_without_reverse_is_rejected():
    import torch
    geo = inputs.Geometry(nkz=3, nqz=3, ne=8, nw=4, na=6, nb=2)
    neigh = np.array([[1, -1], [2, -1], [0, -1], [4, -1], [5, -1], [3, -1]], dtype=np.int32)  # one-way rings
    inst = inputs.make_instance(geo, 6, neigh=neigh, hermitian_pairs=False)
    dev = to_device(inst)
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=3, nqz=3, ne=8, nw=4, mode="mixed")
    Dfull = torch.zeros((3, 4, 6, 3, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(sse.SSEError) as e:
        plan.dtilde(Dfull, torch.empty_like(dev["D_gt"]))
    assert e.value.status == sse.SSE_E_INVALID_ARG and "reverse" in str(e.value)
    S = torch.empty_like(dev["G_gt"])
    with pytest.raises(sse.SSEError):
        plan.execute_full(dev["G_gt"], None, Dfull, None, S, None)
    with pytest.raises(sse.SSEError):  # Sigma^R needs both signs
        plan.execute_full(dev["G_gt"], None, Dfull, None, S, None, S_r=torch.empty_like(S))
    plan.close()
