"""sse_execute_host: the same computation from host buffers.  With both signs the second
sign's copies overlap the first sign's kernels on a second stream; the result must be the
device path's, bit for bit, and within the mixed tolerance of the oracle (Eq. 3)."""
import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs
from tests.gpu_helpers import rel_fro, to_device

pytestmark = pytest.mark.gpu
TOL = 2e-5


def _plan(inst, mode):
    from paper_1912_08810_gb300 import sse
    dev = to_device(inst)
    nkz, ne, na = inst["G_gt"].shape[:3]
    nqz, nw = inst["D_gt"].shape[:2]
    return sse.Plan(dev["neigh"], dev["dH"], nkz=nkz, nqz=nqz, ne=ne, nw=nw, mode=mode), dev


def _device_run(plan, dev, signs):
    import torch
    S = {s: (torch.empty_like(dev["G_" + s]) if s in signs else None) for s in ("gt", "lt")}
    plan.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    torch.cuda.synchronize()
    return {s: S[s].cpu().numpy() for s in signs}


def _host_run(plan, inst, signs, pinned):
    import torch
    h = {k: torch.from_numpy(np.ascontiguousarray(inst[k])) for k in ("G_gt", "G_lt", "D_gt", "D_lt")}
    if pinned:
        h = {k: v.pin_memory() for k, v in h.items()}
    S = {}
    for s in ("gt", "lt"):
        if s in signs:
            t = torch.full_like(h["G_" + s], float("nan"))
            S[s] = t.pin_memory() if pinned else t
        else:
            S[s] = None
    plan.execute_host(h["G_gt"], h["G_lt"], h["D_gt"], h["D_lt"], S["gt"], S["lt"])
    return {s: S[s].numpy() for s in signs}


@pytest.mark.parametrize("geo,seed", [(inputs.TINY, 0),
                                      (inputs.Geometry(nkz=5, nqz=5, ne=29, nw=8, na=6, nb=4), 7)])
def test_host_both_signs_equal_device_path(geo, seed):
    inst = inputs.make_instance(geo, seed)
    plan, dev = _plan(inst, "mixed")
    try:
        ref_dev = _device_run(plan, dev, ("gt", "lt"))
        for pinned in (True, False):
            out = _host_run(plan, inst, ("gt", "lt"), pinned)
            for s in ("gt", "lt"):
                assert np.array_equal(out[s], ref_dev[s])
        plan.status()
        for s in ("gt", "lt"):
            ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], omega_first=1)
            assert rel_fro(out[s], ref) <= TOL
    finally:
        plan.close()


@pytest.mark.parametrize("sign", ["gt", "lt"])
def test_host_one_sign(sign):
    inst = inputs.make_instance(inputs.TINY, 1)
    plan, dev = _plan(inst, "mixed")
    try:
        out = _host_run(plan, inst, (sign,), pinned=True)
        ref_dev = _device_run(plan, dev, (sign,))
        assert np.array_equal(out[sign], ref_dev[sign])
    finally:
        plan.close()


def test_host_fp64_form():
    inst = inputs.make_instance(inputs.TINY, 2)
    plan, dev = _plan(inst, "fp64")
    try:
        out = _host_run(plan, inst, ("gt", "lt"), pinned=True)
        for s in ("gt", "lt"):
            ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], omega_first=1)
            assert rel_fro(out[s], ref) <= 1e-11
    finally:
        plan.close()
