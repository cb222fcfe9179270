"""Batched form: many uneven instances in one persistent launch (sse_execute_batch).

Checks: every instance against the CPU oracle (mixed tolerance 2e-5); bit-identity with
the same instance evaluated alone by sse_execute (the result of an instance does not
depend on what else is in the batch); the autotuner's cached choice; capture of the
batched launch in a CUDA graph; rejection of inconsistent batches."""
import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, to_device

pytestmark = pytest.mark.gpu
TOL = 2e-5


def small_batch(n=6, seed=11):
    spec = inputs.BatchedSpec(n_instances=n, na_range=(8, 40), ne_range=(9, 70), nkz=3, nw=16)
    return inputs.make_batched(spec, seed)


def setup(insts, mode="mixed", signs=("gt", "lt")):
    import torch
    plans, ios, keep = [], [], []
    for inst in insts:
        g = inst["geometry"]
        dev = to_device(inst)
        S = {s: (torch.full_like(dev["G_gt"], float("nan")) if s in signs else None) for s in ("gt", "lt")}
        p = sse.Plan(dev["neigh"], dev["dH"], nkz=g.nkz, nqz=g.nqz, ne=g.ne, nw=g.nw, mode=mode)
        io = p._io(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
        plans.append(p)
        ios.append(io)
        keep.append((dev, S))
    return plans, ios, keep


def test_batch_matches_oracle_and_single_runs():
    import torch
    insts = small_batch()
    plans, ios, keep = setup(insts)
    stream = torch.cuda.current_stream().cuda_stream
    sse.sse_execute_batch([p.handle for p in plans], ios, stream)
    torch.cuda.synchronize()
    plans[0].status()
    assert sse.sse_batch_tuning([p.handle for p in plans], ios) is not None
    for inst, (dev, S) in zip(insts, keep):
        for s in ("gt", "lt"):
            ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"])
            assert rel_fro(S[s].cpu().numpy(), ref) <= TOL
    # the same instances alone: bit-identical
    for p, inst, (dev, S) in zip(plans, insts, keep):
        alone = {s: torch.full_like(S[s], float("nan")) for s in ("gt", "lt")}
        p.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], alone["gt"], alone["lt"])
        torch.cuda.synchronize()
        for s in ("gt", "lt"):
            assert torch.equal(alone[s], S[s])


def test_batch_single_sign_and_second_call_reuses_tuning():
    import torch
    insts = small_batch(n=4, seed=12)
    plans, ios, keep = setup(insts, signs=("lt",))
    stream = torch.cuda.current_stream().cuda_stream
    handles = [p.handle for p in plans]
    sse.sse_execute_batch(handles, ios, stream)
    first = sse.sse_batch_tuning(handles, ios)
    sse.sse_execute_batch(handles, ios, stream)
    torch.cuda.synchronize()
    assert sse.sse_batch_tuning(handles, ios) == first
    for inst, (dev, S) in zip(insts, keep):
        ref = oracle.sigma_atoms(inst["G_lt"], inst["D_lt"], inst["dH"], inst["neigh"])
        assert rel_fro(S["lt"].cpu().numpy(), ref) <= TOL


def test_batch_captured_in_a_cuda_graph():
    import torch
    insts = small_batch(n=3, seed=13)
    plans, ios, keep = setup(insts)
    handles = [p.handle for p in plans]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        sse.sse_execute_batch(handles, ios, side.cuda_stream)  # tunes outside the capture
    torch.cuda.synchronize()
    ref = [{s: S[s].clone() for s in S} for _, S in keep]
    for _, S in keep:
        for s in S:
            S[s].fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        sse.sse_execute_batch(handles, ios, side.cuda_stream)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for r, (_, S) in zip(ref, keep):
        for s in S:
            assert torch.equal(r[s], S[s])


def test_batch_rejects_inconsistent_plans():
    import torch
    a = small_batch(n=1, seed=14)[0]
    geo = inputs.Geometry(nkz=5, nqz=5, ne=12, nw=16, na=8, nb=4)
    b = inputs.make_instance(geo, 1, dtype=np.complex64)
    b["geometry"] = geo
    plans, ios, keep = setup([a, b])
    with pytest.raises(sse.SSEError) as e:
        sse.sse_execute_batch([p.handle for p in plans], ios, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == sse.SSE_E_INVALID_ARG
    plans64, ios64, keep64 = setup([a], mode="fp64")
    with pytest.raises(sse.SSEError):
        sse.sse_execute_batch([p.handle for p in plans64], ios64, torch.cuda.current_stream().cuda_stream)


def test_batched_workload_at_full_size():
    """The batched workload itself (64 instances, Na ~ U[64,1024], NE ~ U[64,512], Nkz=Nqz=3,
    Nw=16, 3..8 random neighbours, complex64, seed 3; about 139 GB of G and Sigma), evaluated
    in one persistent launch and checked per instance against the oracle: the four smallest
    instances in full and the largest on its first and last 16 atoms, both signs; every
    instance's output finite and zero at E = 0."""
    import torch
    spec = inputs.BatchedSpec()
    insts = inputs.make_batched_torch(spec, 3)
    plans, ios, outs = [], [], []
    for inst in insts:
        g = inst["geometry"]
        S = {s: torch.full_like(inst["G_gt"], float("nan")) for s in ("gt", "lt")}
        p = sse.Plan(inst["neigh"], inst["dH"], nkz=g.nkz, nqz=g.nqz, ne=g.ne, nw=g.nw, mode="mixed")
        ios.append(p._io(inst["G_gt"], inst["G_lt"], inst["D_gt"], inst["D_lt"], S["gt"], S["lt"]))
        plans.append(p)
        outs.append(S)
    stream = torch.cuda.current_stream().cuda_stream
    sse.sse_execute_batch([p.handle for p in plans], ios, stream)
    torch.cuda.synchronize()
    plans[0].status()
    for S in outs:
        for s in ("gt", "lt"):
            assert bool(torch.isfinite(torch.view_as_real(S[s])).all())
            assert bool((S[s][:, 0] == 0).all())
    pts = [inst["geometry"].points() for inst in insts]
    order = list(np.argsort(pts))
    for i in order[:4] + order[-1:]:
        inst = insts[i]
        host = {k: inst[k].cpu().numpy() for k in ("G_gt", "G_lt", "D_gt", "D_lt", "dH", "neigh")}
        na = inst["geometry"].na
        ranges = [(0, na)] if i != order[-1] else [(0, 16), (na - 16, na)]
        for s in ("gt", "lt"):
            got = outs[i][s].cpu().numpy()
            for a0, a1 in ranges:
                ref = oracle.sigma_atoms(host["G_" + s], host["D_" + s], host["dH"], host["neigh"], a0, a1)
                assert rel_fro(got[:, :, a0:a1], ref) <= TOL, (i, s, a0)
    for p in plans:
        p.close()
    del insts, outs
    torch.cuda.empty_cache()
