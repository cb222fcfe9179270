"""Kernel timing of a plan (sse_plan_set_timing / sse_plan_timing): events around the
workspace pass and the main kernel of each sse_execute while enabled, none otherwise."""
import numpy as np
import pytest

from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nkz,mode", [(5, "mixed"), (3, "mixed"), (3, "fp64")])
def test_timing_counts_calls_and_splits_the_workspace_pass(nkz, mode):
    import torch
    geo = inputs.Geometry(nkz=nkz, nqz=nkz, ne=24, nw=8, na=6, nb=4)
    inst = inputs.make_instance(geo, 5)
    dev = to_device(inst)
    S = {s: torch.empty_like(dev["G_gt"]) for s in ("gt", "lt")}
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=geo.nkz, nqz=geo.nqz, ne=geo.ne, nw=geo.nw, mode=mode)
    run = lambda: plan.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    run()  # untimed
    sse.sse_plan_set_timing(plan.handle, True)
    for _ in range(3):
        run()
    prep, main, calls = sse.sse_plan_timing(plan.handle)
    assert calls == 3 and main > 0.0 and prep >= 0.0
    if mode == "mixed" and nkz == 5:
        assert prep > 0.0  # the tensor-core form's workspace pass
    sse.sse_plan_set_timing(plan.handle, False)
    run()
    assert sse.sse_plan_timing(plan.handle)[2] == 0  # disabling zeroes and stops
    # more calls than the event ring holds
    sse.sse_plan_set_timing(plan.handle, True)
    for _ in range(70):
        run()
    assert sse.sse_plan_timing(plan.handle)[2] == 70
    plan.status()
