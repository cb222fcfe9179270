"""The bounds-checked build (libsse_gb300_bc.so, compiled with -DSSE_BOUNDS_CHECK): every
kernel family runs through it on small cases -- the FP64 form, both tensor-core forms, the
chain from the full phonon tensor, the pre-combination and retarded kernels, Pi, the
batched launch and the no-alloc entry -- and must report no index outside its buffers
(status SSE_OK, never SSE_E_BOUNDS) while matching the oracle.  It runs in a child process
because a process loads one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path.insert(0, os.environ["TEST_ROOT"])
import numpy as np, torch
import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, to_device
assert sse.load()._name.endswith("libsse_gb300_bc.so")

def plan_for(dev, geo, mode):
    return sse.Plan(dev["neigh"], dev["dH"], nkz=geo.nkz, nqz=geo.nqz, ne=geo.ne, nw=geo.nw, mode=mode)

for mode, geo, dt, tol in (("fp64", inputs.Geometry(nkz=3, nqz=2, ne=20, nw=4, na=7, nb=4), np.complex128, 1e-11),
                           ("mixed", inputs.Geometry(nkz=3, nqz=3, ne=45, nw=16, na=9, nb=4), np.complex64, 2e-5),
                           ("mixed", inputs.Geometry(nkz=5, nqz=5, ne=27, nw=32, na=6, nb=4), np.complex128, 2e-5)):
    inst = inputs.make_instance(geo, 3, dtype=dt)
    full = inputs.make_phonon_full(geo, 4, inst["neigh"], dtype=dt)
    dev = to_device(inst)
    for k in full:
        dev[k] = torch.from_numpy(full[k]).cuda()
    p = plan_for(dev, geo, mode)
    S = {s: torch.full_like(dev["G_gt"], float("nan")) for s in ("gt", "lt", "r")}
    p.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    torch.cuda.synchronize(); p.status()
    for s in ("gt", "lt"):
        ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"])
        assert rel_fro(S[s].cpu().numpy(), ref) <= tol, (mode, s)
    p.execute_full(dev["G_gt"], dev["G_lt"], dev["D_gt_full"], dev["D_lt_full"], S["gt"], S["lt"], S["r"])
    Dt = torch.empty_like(dev["D_gt"])
    p.dtilde(dev["D_gt_full"], Dt)
    torch.cuda.synchronize(); p.status()
    ref = oracle.sigma_atoms(inst["G_gt"], oracle.dtilde(full["D_gt_full"], inst["neigh"]), inst["dH"], inst["neigh"])
    assert rel_fro(S["gt"].cpu().numpy(), ref) <= tol
    pis = torch.empty((geo.nqz, geo.nw, geo.na, geo.nb + 1, 3, 3), dtype=dev["G_gt"].dtype, device="cuda")
    p.pi(dev["G_gt"], dev["G_lt"], pis, None)
    torch.cuda.synchronize(); p.status()
    ref = oracle.pi(inst["G_gt"], inst["G_lt"], inst["dH"], inst["neigh"], geo.nqz, geo.nw)
    assert rel_fro(pis.cpu().numpy(), ref) <= (1e-11 if dt == np.complex128 else 1e-6)
    if mode == "mixed":
        io = p._io(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
        sse.sse_execute_batch([p.handle], [io], torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize(); p.status()
        g = sse.sse_geometry(geo.nkz, geo.nqz, geo.ne, geo.nw, geo.na, geo.nb, 12, 1, dev["neigh"].data_ptr(),
                             dev["dH"].data_ptr(), sse.SSE_C128 if dt == np.complex128 else sse.SSE_C64, sse.SSE_MODE_MIXED)
        sse.sse_execute_noalloc(g, io, torch.cuda.current_stream().cuda_stream)
        ref = oracle.sigma_atoms(inst["G_lt"], inst["D_lt"], inst["dH"], inst["neigh"])
        assert rel_fro(S["lt"].cpu().numpy(), ref) <= tol
    p.close()
print("bounds-checked build: ok")
"""


def test_bounds_checked_build_runs_clean():
    lib = os.path.join(ROOT, "paper_1912_08810_gb300", "libsse_gb300_bc.so")
    if not os.path.exists(lib):
        from paper_1912_08810_gb300 import build
        build.build(bounds_check=True)
    env = dict(os.environ, SSE_GB300_LIB=lib, TEST_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "bounds-checked build: ok" in r.stdout
