"""Helpers shared by the GPU tests: run one problem through libtsu and through the oracle on the
same seeded inputs, and compare."""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from paper_2005_11931_gb300 import inputs, tsu


def relerr(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_tau(ext, g) -> float:
    return 0.4 * min(g.dx, g.dy) / math.sqrt(max(ext[1], ext[3]))


def run_gpu(n, depth, u0_np, steps, dtype="f32", form=tsu.TSU_FORM_STANDARD, ny=None, rec_ij=None, tau=None,
            energy=True, rows=0, kernel=0, tdepth=0):
    """Taylor start + (steps-1) steps + observe.  Returns dict(u, u_prev, energy[steps], traces[steps][nrec],
    tau, ext, sim)."""
    sim = tsu.Simulation.create(n, depth, dtype=dtype, form=form, ny=ny, tau=tau)
    g = sim.g
    tdt = tsu.DTYPES[sim.dtype]
    u0 = torch.zeros((g.ny, g.ld), dtype=tdt, device="cuda")
    u0[:, : g.nx] = torch.from_numpy(np.ascontiguousarray(u0_np[:, : g.nx])).to(tdt)
    sim.init(u0)
    e = torch.zeros(max(steps, 1), dtype=torch.float64, device="cuda") if energy else None
    rec = tr = None
    if rec_ij is not None:
        rec = torch.from_numpy(inputs.flat_index(rec_ij, g.ld)).cuda()
        tr = torch.zeros((steps, len(rec_ij)), dtype=tdt, device="cuda")
    if steps > 1:
        sim.step(steps - 1, energy=e[: steps - 1] if energy else None, rec_idx=rec,
                 traces=tr[: steps - 1] if tr is not None else None, rows=rows, kernel=kernel, tdepth=tdepth)
    sim.observe(energy=e[steps - 1:] if energy else None, rec_idx=rec, trace=tr[steps - 1] if tr is not None else None)
    torch.cuda.synchronize()
    up = sim.u_prev if sim.u_prev is not None else sim.u - sim.v
    return dict(u=sim.u[:, : g.nx].double().cpu().numpy(), u_prev=up[:, : g.nx].double().cpu().numpy(),
                energy=e.cpu().numpy() if energy else None, traces=tr.double().cpu().numpy() if tr is not None else None,
                tau=sim.tau, ext=sim.ext, sim=sim)


def run_oracle(n, depth, u0_np, steps, ny=None, rec_ij=None, tau=None, energy=True):
    g = oracle.grid(n, ny or n)
    hx, hy, ext = oracle.make_depth(g, depth)
    if tau is None:
        tau = oracle_tau(ext, g)
    rec = inputs.flat_index(rec_ij, g.ld) if rec_ij is not None else None
    out = oracle.forward(g, tau, hx, hy, np.ascontiguousarray(u0_np[:, : g.nx]), None, steps, want_energy=energy,
                         rec_idx=rec)
    out["tau"] = tau
    out["ext"] = ext
    return out
