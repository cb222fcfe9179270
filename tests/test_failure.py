"""Failure detection without a GPU fault: bounded device waits that run out, cancelled
requests, injected allocation failures.

The stall hook (sse_debug_inject(SSE_INJECT_STALL)) leaves one copy of each CTA's first
work unit unissued, so a wait on a barrier that nothing completes runs out its bound.
The kernel must then drain what it has in flight, free its tensor memory and return;
the timeout must reach the caller as SSE_E_TIMEOUT (sse_plan_status, sse_poll); and the
next call on the same plan must be correct.  No test here faults, traps or hangs a GPU."""
import time

import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, to_device

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(autouse=True)
def disarm():
    yield
    sse.sse_debug_inject(sse.SSE_INJECT_NONE)


def make(inst, mode="mixed"):
    import torch
    dev = to_device(inst)
    nkz, ne, na = inst["G_gt"].shape[:3]
    nqz, nw = inst["D_gt"].shape[:2]
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=nkz, nqz=nqz, ne=ne, nw=nw, mode=mode)
    S = {s: torch.full_like(dev["G_gt"], float("nan")) for s in ("gt", "lt")}
    return plan, dev, S


def execute(plan, dev, S):
    plan.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])


@pytest.mark.parametrize("geo", [
    inputs.Geometry(nkz=5, nqz=5, ne=40, nw=32, na=12, nb=4),  # warp-specialised form
    inputs.Geometry(nkz=3, nqz=3, ne=48, nw=4, na=16, nb=4),   # single-role form
])
def test_stalled_wait_times_out_then_plan_recovers(geo):
    import torch
    inst = inputs.make_instance(geo, 5)
    plan, dev, S = make(inst)
    sse.sse_debug_inject(sse.SSE_INJECT_STALL)
    t0 = time.time()
    execute(plan, dev, S)
    torch.cuda.synchronize()  # the kernel returned: every wait is bounded
    assert time.time() - t0 < 30.0
    with pytest.raises(sse.SSEError) as e:
        plan.status()
    assert e.value.status == sse.SSE_E_TIMEOUT
    plan.status()  # the word was cleared by the read
    execute(plan, dev, S)  # the hook is one-shot
    torch.cuda.synchronize()
    plan.status()
    for s in ("gt", "lt"):
        ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"])
        assert rel_fro(S[s].cpu().numpy(), ref) <= TOL


def test_stalled_batch_reports_timeout_on_plans0():
    import torch
    spec = inputs.BatchedSpec(n_instances=3, na_range=(8, 24), ne_range=(20, 40), nkz=3, nw=16)
    insts = inputs.make_batched(spec, 31)
    made = [make(i) for i in insts]
    handles = [p.handle for p, _, _ in made]
    ios = [p._io(d["G_gt"], d["G_lt"], d["D_gt"], d["D_lt"], S["gt"], S["lt"]) for p, d, S in made]
    stream = torch.cuda.current_stream().cuda_stream
    sse.sse_execute_batch(handles, ios, stream)  # tunes once, untouched by the hook
    torch.cuda.synchronize()
    sse.sse_debug_inject(sse.SSE_INJECT_STALL)
    sse.sse_execute_batch(handles, ios, stream)
    torch.cuda.synchronize()
    with pytest.raises(sse.SSEError) as e:
        made[0][0].status()
    assert e.value.status == sse.SSE_E_TIMEOUT
    sse.sse_execute_batch(handles, ios, stream)
    torch.cuda.synchronize()
    made[0][0].status()
    for inst, (_, _, S) in zip(insts, made):
        ref = oracle.sigma_atoms(inst["G_lt"], inst["D_lt"], inst["dH"], inst["neigh"])
        assert rel_fro(S["lt"].cpu().numpy(), ref) <= TOL


def poll_until(server, ticket, pred, limit_s=60.0):
    t0 = time.time()
    while True:
        rc, r = sse.sse_poll(server, ticket)
        if pred(rc, r):
            return rc, r
        assert time.time() - t0 < limit_s, "server made no progress"
        time.sleep(0.0005)


def server_request(seed, na, ne):
    import torch
    geo = inputs.Geometry(nkz=3, nqz=3, ne=ne, nw=16, na=na, nb=8)
    rng = np.random.default_rng(seed)
    neigh = inputs.random_neighbours(rng, na, 8)
    inst = inputs.make_instance(geo, seed, dtype=np.complex64, neigh=neigh, hermitian_pairs=False)
    plan, dev, S = make(inst)
    io = plan._io(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    return dict(inst=inst, plan=plan, dev=dev, S=S, io=io)


def test_stalled_round_times_out_every_ticket_of_that_round():
    """Two long rounds hold both server streams; three requests submitted meanwhile form one
    round, which the stall hook hits: each of its tickets reports SSE_E_TIMEOUT, the long
    rounds report SSE_OK, and the same three requests are correct when resubmitted."""
    import torch
    blockers = [server_request(40 + i, 512, 256) for i in range(2)]
    small = [server_request(50 + i, 24, 40) for i in range(3)]
    torch.cuda.synchronize()
    server = sse.sse_server_create(1 << 40, 16, 20000)
    try:
        tb = []
        for b in blockers:
            t = sse.sse_submit(server, b["plan"].handle, b["io"])
            poll_until(server, t, lambda rc, r: rc != sse.SSE_NOT_READY or r.t_start_ms > 0)
            tb.append(t)
        sse.sse_debug_inject(sse.SSE_INJECT_STALL)
        ts = [sse.sse_submit(server, q["plan"].handle, q["io"]) for q in small]
        res = {t: poll_until(server, t, lambda rc, r: rc != sse.SSE_NOT_READY) for t in tb + ts}
        stalled = [res[t] for t in ts]
        assert all(rc == sse.SSE_E_TIMEOUT for rc, _ in stalled), [rc for rc, _ in stalled]
        assert len({r.t_start_ms for _, r in stalled}) == 1 and stalled[0][1].round_size == 3
        assert all(res[t][0] == sse.SSE_OK for t in tb)
        ts2 = [sse.sse_submit(server, q["plan"].handle, q["io"]) for q in small]
        for t in ts2:
            rc, _ = poll_until(server, t, lambda rc, r: rc != sse.SSE_NOT_READY)
            assert rc == sse.SSE_OK
    finally:
        sse.sse_server_destroy(server)
    for q in small:
        for s in ("gt", "lt"):
            inst = q["inst"]
            ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"])
            assert rel_fro(q["S"][s].cpu().numpy(), ref) <= TOL


def test_shutdown_cancels_what_never_started():
    import torch
    reqs = [server_request(60 + i, 256, 128) for i in range(5)]
    torch.cuda.synchronize()
    server = sse.sse_server_create(1 << 40, 1, 20000)  # one request admitted at a time
    try:
        tickets = [sse.sse_submit(server, q["plan"].handle, q["io"]) for q in reqs]
        poll_until(server, tickets[0], lambda rc, r: rc != sse.SSE_NOT_READY or r.t_start_ms > 0)
        sse.sse_server_shutdown(server)
        with pytest.raises(sse.SSEError) as e:
            sse.sse_submit(server, reqs[0]["plan"].handle, reqs[0]["io"])
        assert e.value.status == sse.SSE_E_SHUTDOWN
        codes = [sse.sse_poll(server, t)[0] for t in tickets]
    finally:
        sse.sse_server_destroy(server)
    assert codes[0] == sse.SSE_OK
    assert codes[-1] == sse.SSE_E_CANCELLED
    assert all(c in (sse.SSE_OK, sse.SSE_E_CANCELLED) for c in codes)
    ran = [c == sse.SSE_OK for c in codes]
    assert ran == sorted(ran, reverse=True)  # arrival order: a prefix ran, the rest was cancelled


def test_injected_allocation_failures_are_codes():
    import torch
    geo = inputs.Geometry(nkz=5, nqz=5, ne=16, nw=8, na=6, nb=4)
    inst = inputs.make_instance(geo, 3)
    dev = to_device(inst)
    sse.sse_debug_inject(sse.SSE_INJECT_ALLOC_FAIL)
    with pytest.raises(sse.SSEError) as e:  # the tensor-core workspace
        sse.Plan(dev["neigh"], dev["dH"], nkz=5, nqz=5, ne=16, nw=8, mode="mixed")
    assert e.value.status == sse.SSE_E_OUT_OF_MEMORY
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=5, nqz=5, ne=16, nw=8, mode="mixed")  # one-shot
    S = {s: torch.empty_like(dev["G_gt"]) for s in ("gt", "lt")}
    io = plan._io(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    stream = torch.cuda.current_stream().cuda_stream
    sse.sse_debug_inject(sse.SSE_INJECT_ALLOC_FAIL)
    with pytest.raises(sse.SSEError) as e:  # the batched launch's work counter
        sse.sse_execute_batch([plan.handle], [io], stream)
    assert e.value.status == sse.SSE_E_OUT_OF_MEMORY
    sse.sse_execute_batch([plan.handle], [io], stream)
    torch.cuda.synchronize()
    plan.status()
    ref = oracle.sigma_atoms(inst["G_gt"], inst["D_gt"], inst["dH"], inst["neigh"])
    assert rel_fro(S["gt"].cpu().numpy(), ref) <= TOL


def test_admission_counts_the_plan_workspace():
    """A request whose buffers fit the budget but whose plan's workspace does not can
    never be admitted."""
    geo = inputs.Geometry(nkz=5, nqz=5, ne=16, nw=8, na=6, nb=4)
    inst = inputs.make_instance(geo, 4)
    plan, dev, S = make(inst)
    io = plan._io(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    bufs = 2 * 16 * (2 * geo.nkz * geo.ne * geo.na * 144 + geo.nqz * geo.nw * geo.na * geo.nb * 9)
    ws = plan.info().workspace_bytes
    assert ws > 0
    server = sse.sse_server_create(bufs + ws - 1, 4, 5000)
    try:
        with pytest.raises(sse.SSEError) as e:
            sse.sse_submit(server, plan.handle, io)
        assert e.value.status == sse.SSE_E_OVER_BUDGET
    finally:
        sse.sse_server_destroy(server)
    server = sse.sse_server_create(bufs + ws, 4, 5000)
    try:
        t = sse.sse_submit(server, plan.handle, io)
        rc, _ = poll_until(server, t, lambda rc, r: rc != sse.SSE_NOT_READY)
        assert rc == sse.SSE_OK
    finally:
        sse.sse_server_destroy(server)
