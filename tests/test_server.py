"""Serving loop: continuous batching of SSE requests (sse_server_create / sse_submit /
sse_poll / sse_server_destroy).

The central check: a request's result is the same whether it ran alone or mixed into a
round with other requests (bit-for-bit here, well within the mixed tolerance), and it
matches the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1912_08810_gb300 import inputs, sse
from tests.gpu_helpers import rel_fro, to_device

pytestmark = pytest.mark.gpu
TOL = 2e-5


def make_requests(n, seed):
    import torch
    spec = inputs.BatchedSpec(n_instances=n, na_range=(8, 48), ne_range=(9, 60), nkz=3, nw=16)
    insts = inputs.make_batched(spec, seed)
    reqs = []
    for inst in insts:
        g = inst["geometry"]
        dev = to_device(inst)
        S = {s: torch.full_like(dev["G_gt"], float("nan")) for s in ("gt", "lt")}
        plan = sse.Plan(dev["neigh"], dev["dH"], nkz=g.nkz, nqz=g.nqz, ne=g.ne, nw=g.nw, mode="mixed")
        io = plan._io(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
        reqs.append(dict(inst=inst, dev=dev, S=S, plan=plan, io=io))
    return reqs


def wait_all(server, tickets, limit_s=120.0):
    results = {}
    t0 = time.time()
    while len(results) < len(tickets):
        for t in tickets:
            if t in results:
                continue
            rc, r = sse.sse_poll(server, t)
            if rc != sse.SSE_NOT_READY:
                results[t] = (rc, r)
        assert time.time() - t0 < limit_s, "requests did not finish"
        time.sleep(0.002)
    return results


def test_results_same_alone_and_in_the_mix():
    import torch
    torch.cuda.synchronize()
    reqs = make_requests(8, 21)
    server = sse.sse_server_create(1 << 40, 4, 5000)
    try:
        tickets = [sse.sse_submit(server, r["plan"].handle, r["io"]) for r in reqs]
        results = wait_all(server, tickets)
        rounds, nbytes, inflight = sse.sse_server_stats(server)
    finally:
        sse.sse_server_destroy(server)
    assert all(rc == sse.SSE_OK for rc, _ in results.values())
    sizes = [r.round_size for _, r in results.values()]
    assert max(sizes) > 1, "no round mixed several requests"
    assert rounds >= 2 and nbytes == 0 and inflight == 0
    for _, r in results.values():
        assert r.t_submit_ms <= r.t_start_ms <= r.t_end_ms
    for req in reqs:
        mixed = {s: req["S"][s].clone() for s in ("gt", "lt")}
        alone = {s: torch.full_like(mixed[s], float("nan")) for s in ("gt", "lt")}
        d = req["dev"]
        req["plan"].execute(d["G_gt"], d["G_lt"], d["D_gt"], d["D_lt"], alone["gt"], alone["lt"])
        torch.cuda.synchronize()
        for s in ("gt", "lt"):
            assert torch.equal(mixed[s], alone[s])
    for req in reqs[:3]:
        inst = req["inst"]
        for s in ("gt", "lt"):
            ref = oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"])
            assert rel_fro(req["S"][s].cpu().numpy(), ref) <= TOL


def test_budget_limits_admission_and_errors_are_codes():
    reqs = make_requests(3, 22)
    one = None
    for r in reqs:
        g = r["inst"]["geometry"]
        nb = (2 * g.nkz * g.ne * g.na * 144 + g.nqz * g.nw * g.na * g.nb * 9) * 8 * 2
        nb += r["plan"].info().workspace_bytes  # admission also counts what the plan holds
        one = nb if one is None else max(one, nb)
    # a budget for one request at a time: every round holds exactly one request
    server = sse.sse_server_create(one, 8, 5000)
    try:
        tickets = [sse.sse_submit(server, r["plan"].handle, r["io"]) for r in reqs]
        results = wait_all(server, tickets)
        assert all(rc == sse.SSE_OK and r.round_size == 1 for rc, r in results.values())
        rc, _ = sse.sse_poll(server, tickets[0])  # already collected
        assert rc == sse.SSE_E_UNKNOWN_TICKET
        rc, _ = sse.sse_poll(server, 987654321)
        assert rc == sse.SSE_E_UNKNOWN_TICKET
    finally:
        sse.sse_server_destroy(server)
    tiny = sse.sse_server_create(1024, 1, 1000)
    try:
        with pytest.raises(sse.SSEError) as e:
            sse.sse_submit(tiny, reqs[0]["plan"].handle, reqs[0]["io"])
        assert e.value.status == sse.SSE_E_OVER_BUDGET
    finally:
        sse.sse_server_destroy(tiny)


def test_destroy_with_pending_work_returns():
    reqs = make_requests(6, 23)
    server = sse.sse_server_create(1 << 40, 1, 10000)
    tickets = [sse.sse_submit(server, r["plan"].handle, r["io"]) for r in reqs]
    t0 = time.time()
    sse.sse_server_shutdown(server)  # cancels what has not started, drains the rest
    codes = [sse.sse_poll(server, t)[0] for t in tickets]
    sse.sse_server_destroy(server)
    assert time.time() - t0 < 10.0
    assert all(c in (sse.SSE_OK, sse.SSE_E_CANCELLED) for c in codes)
    assert sse.SSE_E_CANCELLED in codes  # one admitted at a time: not all six ran
