"""sse_execute_noalloc: the mixed-mode entry point for callers that cannot let the library
allocate memory (for example a framework whose allocator owns all device memory).

It must give the same Sigma as the planned path (sse_plan + sse_execute, mixed mode) and
match the FP64 oracle, call after call, even though every call reuses the same built-in
scratch array.  This
file is collected last on purpose, so a failure here does not hide any other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, run, to_device

pytestmark = pytest.mark.gpu
TOL = 2e-5  # the mixed path's stated tolerance


def noalloc_call(dev, nkz, nqz, ne, nw, omega_first=1, mode=sse.SSE_MODE_MIXED):
    import torch
    na, nb = dev["neigh"].shape
    dtype = sse.SSE_C128 if dev["dH"].dtype == torch.complex128 else sse.SSE_C64
    geo = sse.sse_geometry(nkz, nqz, ne, nw, na, nb, 12, omega_first, dev["neigh"].data_ptr(),
                           dev["dH"].data_ptr(), dtype, mode)
    S = {s: torch.full_like(dev["G_gt"], float("nan")) for s in ("gt", "lt")}
    io = sse.sse_io(dev["G_gt"].data_ptr(), dev["G_lt"].data_ptr(), dev["D_gt"].data_ptr(),
                    dev["D_lt"].data_ptr(), S["gt"].data_ptr(), S["lt"].data_ptr())
    sse.sse_execute_noalloc(geo, io, torch.cuda.current_stream().cuda_stream)
    return {s: S[s].cpu().numpy() for s in S}


@pytest.mark.parametrize("geo_seed", [
    (inputs.TINY, 0, np.complex128),
    (inputs.Geometry(nkz=5, nqz=5, ne=40, nw=32, na=12, nb=4), 3, np.complex128),
    (inputs.Geometry(nkz=3, nqz=3, ne=33, nw=16, na=10, nb=4), 4, np.complex64),
])
def test_matches_planned_path_on_two_calls_in_a_row(geo_seed):
    geo, seed, dt = geo_seed
    inst = inputs.make_instance(geo, seed, dtype=dt)
    ref = run(inst, "mixed")
    exact = {s: oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"]) for s in ("gt", "lt")}
    dev = to_device(inst)
    for _ in range(2):
        out = noalloc_call(dev, geo.nkz, geo.nqz, geo.ne, geo.nw)
        for s in ("gt", "lt"):
            assert np.all(np.isfinite(out[s]))
            assert rel_fro(out[s], ref[s]) <= TOL
            assert rel_fro(out[s], exact[s]) <= TOL  # and against the FP64 oracle itself


def test_rejects_what_it_cannot_run():
    inst = inputs.make_instance(inputs.Geometry(nkz=6, nqz=6, ne=8, nw=2, na=4, nb=4), 1)
    dev = to_device(inst)
    with pytest.raises(sse.SSEError) as e:
        noalloc_call(dev, 6, 6, 8, 2)
    assert e.value.status == sse.SSE_E_INVALID_ARG and "Nkz <= 5" in str(e.value)
    with pytest.raises(sse.SSEError) as e:
        noalloc_call(dev, 6, 6, 8, 2, mode=sse.SSE_MODE_FP64)
    assert e.value.status == sse.SSE_E_INVALID_ARG


def test_rejects_out_of_range_neighbour_checked_on_device():
    geo = inputs.Geometry(nkz=3, nqz=3, ne=10, nw=4, na=6, nb=4)
    inst = inputs.make_instance(geo, 2)
    dev = to_device(inst)
    dev["neigh"][4, 2] = 6  # one past the last atom
    with pytest.raises(sse.SSEError) as e:
        noalloc_call(dev, geo.nkz, geo.nqz, geo.ne, geo.nw)
    assert e.value.status == sse.SSE_E_INVALID_ARG and "flat index 18" in str(e.value)
    # a good call right after a rejected one still works (the scratch is cleared per call)
    dev["neigh"][4, 2] = 0
    inst["neigh"][4, 2] = 0
    ref = run(inst, "mixed")
    out = noalloc_call(dev, geo.nkz, geo.nqz, geo.ne, geo.nw)
    assert rel_fro(out["gt"], ref["gt"]) <= TOL
