"""Helpers shared by the GPU parity tests: move a seeded instance to the device, run a
plan through the C ABI, and measure errors against the oracle."""
import numpy as np


def to_device(inst):
    import torch
    out = {}
    for k in ("G_gt", "G_lt", "D_gt", "D_lt", "dH", "neigh"):
        out[k] = torch.from_numpy(np.ascontiguousarray(inst[k])).cuda()
    return out


def run(inst, mode="fp64", signs=("gt", "lt"), omega_first=1, plan_out=None):
    """Run one instance through the C ABI; returns {sign: numpy Sigma}."""
    import torch
    from paper_1912_08810_gb300 import sse
    dev = to_device(inst)
    nkz, ne, na = inst["G_gt"].shape[:3]
    nqz, nw = inst["D_gt"].shape[:2]
    plan = sse.Plan(dev["neigh"], dev["dH"], nkz=nkz, nqz=nqz, ne=ne, nw=nw,
                    omega_first=omega_first, mode=mode)
    S = {s: (torch.full_like(dev["G_" + s], float("nan")) if s in signs else None) for s in ("gt", "lt")}
    plan.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"])
    torch.cuda.synchronize()
    plan.status()
    if plan_out is not None:
        plan_out.append(plan)
    else:
        plan.close()
    return {s: S[s].cpu().numpy() for s in signs}


def rel_fro(x, ref):
    n = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (n if n > 0 else 1.0))


def max_block_rel(x, ref):
    """Largest per-block relative error (block = last two axes)."""
    d = np.linalg.norm((x - ref).reshape(-1, ref.shape[-2] * ref.shape[-1]), axis=1)
    n = np.linalg.norm(ref.reshape(-1, ref.shape[-2] * ref.shape[-1]), axis=1)
    scale = max(float(n.max()), 1e-300)
    return float(np.max(d / np.maximum(n, 1e-3 * scale)))
