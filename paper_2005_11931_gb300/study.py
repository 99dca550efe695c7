"""Studies of the eps-regularised family (arXiv:2005.11931 Sec. 3.2), built on the library's entry
points: every solve, field comparison and derivative runs in libtsu's kernels; this module only
sets problems up and reads back scalars and receiver traces.

- ``eps_convergence``: the family u_eps for a halving sequence of widths, advanced together by
  ``tsu_batch_run`` to one common time, and the relative differences of neighbours (the paper's
  claim that the family is Cauchy as eps -> 0).
- ``mollifier_gap``: the same problem regularised with the Gaussian and with the Friedrichs
  mollifier at each width (the limit does not depend on the mollifier).
- ``reflected_pulse``: receiver traces between a source and a line singularity, with the
  incident and the reflected pulse picked out.
- ``misfit_eps_gradient``: J = 1/2 sum (u(receivers) - observed)^2 and dJ/deps, the forward and
  adjoint face gradients chained through d h_eps / d eps.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import inputs, tsu

KINDS = {
    "line_x": [(inputs.LINE_X, 1, 1.0, 0.5, 0.5)],
    "line_y": [(inputs.LINE_Y, 1, 1.0, 0.5, 0.5)],
    "point": [(inputs.POINT, 1, 0.01, 0.5, 0.5)],
    "line_point": [(inputs.LINE_X, 1, 1.0, 0.5, 0.5), (inputs.POINT, 1, 0.01, 0.5, 0.5)],
}


def _norms(sim_a, sim_b, ws) -> tuple[float, float]:
    out = torch.zeros(2, dtype=torch.float64, device=sim_a.u.device)
    tsu.tsu_diff_norms(sim_a.g, sim_a.dtype, sim_a.u, sim_b.u, out, ws)
    d, b = out.cpu().numpy()
    return float(d), float(b)


def _family(depths, n, T, u0_spec, form=tsu.TSU_FORM_INCREMENT):
    """FP32 simulations of ``depths`` on one n x n grid, one common tau (the smallest the CFL rule
    allows over the family) and the step count reaching time T; all advanced by tsu_batch_run."""
    sims = [tsu.Simulation.create(n, d, dtype="f32", form=form) for d in depths]
    tau = min(s.tau for s in sims)
    sims = [tsu.Simulation.create(n, d, dtype="f32", form=form, tau=tau) for d in depths]
    steps = max(2, int(math.ceil(T / tau)))
    x0, y0, w, a = u0_spec
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, sims[0].g.ld, x0, y0, w, a, np.float32)).cuda()
    for s in sims:
        s.init(u0)
    nsteps = [steps - 1] * len(sims)
    wsb = tsu.tsu_batch_workspace(sims, nsteps)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_batch_run(sims, nsteps, ws, wsb)
    tsu.tsu_sync_status(ws, wsb)
    return sims, tau, steps


def eps_convergence(kind: str, eps_list, n: int = 1025, T: float = 0.15,
                    u0_spec=(0.40, 0.5, 0.03, 1.0)) -> dict:
    """Relative differences ||u_{eps_k} - u_{eps_{k+1}}|| / ||u_{eps_{k+1}}|| at time T for the
    family of one singularity kind (Gaussian mollifier, background 1)."""
    depths = [dict(background=1.0, eps=float(e), mollifier=inputs.GAUSS, sings=KINDS[kind]) for e in eps_list]
    sims, tau, steps = _family(depths, n, T, u0_spec)
    ws = torch.empty(tsu.tsu_reduce_workspace(), dtype=torch.uint8, device="cuda")
    rel = []
    for a, b in zip(sims[:-1], sims[1:]):
        d, nb = _norms(a, b, ws)
        rel.append(math.sqrt(d / nb))
    return {"kind": kind, "eps": [float(e) for e in eps_list], "n": n, "tau": tau, "steps": steps, "T": steps * tau,
            "relative_differences": rel}


def mollifier_gap(eps_list, n: int = 1025, T: float = 0.15, kind: str = "line_x",
                  u0_spec=(0.40, 0.5, 0.03, 1.0)) -> dict:
    """||u_Gauss - u_Friedrichs|| / ||u_Friedrichs|| at time T for each width (same problem, same
    tau, the two mollifiers of Sec. 3.1)."""
    depths = []
    for e in eps_list:
        for moll in (inputs.GAUSS, inputs.FRIEDRICHS):
            depths.append(dict(background=1.0, eps=float(e), mollifier=moll, sings=KINDS[kind]))
    sims, tau, steps = _family(depths, n, T, u0_spec)
    ws = torch.empty(tsu.tsu_reduce_workspace(), dtype=torch.uint8, device="cuda")
    gaps = []
    for k in range(len(eps_list)):
        d, nb = _norms(sims[2 * k], sims[2 * k + 1], ws)
        gaps.append(math.sqrt(d / nb))
    return {"kind": kind, "eps": [float(e) for e in eps_list], "n": n, "tau": tau, "steps": steps, "T": steps * tau,
            "relative_gaps": gaps}


def reflected_pulse(eps: float, n: int = 769, T: float = 0.45, amp: float = 1.0, x_src: float = 0.30,
                    x_rec: float = 0.40, width: float = 0.03) -> dict:
    """A hump at (x_src, 0.5), a line singularity amp phi_eps(x - 0.5) on background 1 and a
    receiver at (x_rec, 0.5) between them.  The same run without the singularity (same tau) gives
    the free wave; the difference of the two receiver traces is the wave the line sends back.
    Returns the free wave's peak and arrival and the reflected wave's signed peak and arrival."""
    line = dict(background=1.0, eps=float(eps), mollifier=inputs.GAUSS, sings=[(inputs.LINE_X, 1, amp, 0.5, 0.5)])
    free = dict(background=1.0, eps=float(eps), mollifier=inputs.GAUSS, sings=[])
    sim = tsu.Simulation.create(n, line, dtype="f32")
    ref = tsu.Simulation.create(n, free, dtype="f32", tau=sim.tau)
    steps = max(2, int(math.ceil(T / sim.tau)))
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, sim.g.ld, x_src, 0.5, width, 1.0, np.float32)).cuda()
    i, j = round(x_rec * (n - 1)), round(0.5 * (n - 1))
    rec = torch.tensor([j * sim.g.ld + i], dtype=torch.int64, device="cuda")
    traces = []
    for s in (sim, ref):
        tr = torch.zeros((steps, 1), dtype=torch.float32, device="cuda")
        s.init(u0)
        s.step(steps - 1, rec_idx=rec, traces=tr[: steps - 1])
        s.observe(rec_idx=rec, trace=tr[steps - 1])
        traces.append(tr[:, 0].double().cpu().numpy())
    t = sim.tau * np.arange(1, steps + 1)
    scattered = traces[0] - traces[1]
    inc = int(np.argmax(np.abs(traces[1])))
    rfl = int(np.argmax(np.abs(scattered)))
    return {"eps": float(eps), "n": n, "tau": sim.tau, "steps": steps, "trace": traces[0], "free_trace": traces[1],
            "incident_peak": float(traces[1][inc]), "incident_arrival": float(t[inc]),
            "reflected_peak": float(scattered[rfl]), "reflected_arrival": float(t[rfl])}


def misfit_eps_gradient(n: int, depth: dict, u0: np.ndarray, S: int, rec_ij: np.ndarray, eps_obs: float,
                        dtype: str = "f64", ckpt_every: int = 64) -> dict:
    """J(eps) = 1/2 sum_n sum_r (u^n(rec_r) - d^n_r)^2 with observations d from the same problem at
    eps_obs, and dJ/deps = sum_faces (dJ/dhx dhx/deps + dJ/dhy dhy/deps): forward with traces and
    checkpoints, tsu_adjoint, then tsu_depth_eps_gradient.  Same tau for both runs."""
    form = tsu.TSU_FORM_STANDARD if dtype == "f64" else tsu.TSU_FORM_INCREMENT
    sim = tsu.Simulation.create(n, depth, dtype=dtype, form=form)
    g, tdt = sim.g, tsu.DTYPES[sim.dtype]
    obs_sim = tsu.Simulation.create(n, dict(depth, eps=float(eps_obs)), dtype=dtype, form=form, tau=sim.tau)
    u0p = np.zeros((g.ny, g.ld))
    u0p[:, :n] = u0[:, :n]
    u0d = torch.from_numpy(u0p).to(tdt).cuda()
    rec = torch.from_numpy(inputs.flat_index(rec_ij, g.ld)).cuda()
    nrec = rec.numel()

    def run(s, traces, ck=None):
        s.init(u0d)
        if S > 1:
            s.step(S - 1, rec_idx=rec, traces=traces[: S - 1], ckpt=ck, ckpt_every=ckpt_every if ck is not None else 0)
        s.observe(rec_idx=rec, trace=traces[S - 1])

    obs = torch.zeros((S, nrec), dtype=tdt, device="cuda")
    run(obs_sim, obs)
    tr = torch.zeros((S, nrec), dtype=tdt, device="cuda")
    slots = max(tsu.tsu_ckpt_slots(S, ckpt_every), 1)
    ck = torch.zeros((slots, 2, g.ny, g.ld), dtype=tdt, device="cuda")
    run(sim, tr, ck)
    res = tr - obs
    gx = torch.zeros((g.ny, g.ld), dtype=torch.float64, device="cuda")
    gy = torch.zeros_like(gx)
    gu0 = torch.zeros((g.ny, g.ld), dtype=tdt, device="cuda")
    gu1 = torch.zeros_like(gu0)
    wsb = tsu.tsu_adjoint_workspace(g, sim.dtype, form, S, ckpt_every, nrec)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_adjoint(g, sim.dtype, form, sim.tau, sim.medium, S, ckpt_every, ck, u0d, rec, res, gx, gy, gu0, gu1, ws,
                    wsb)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rws = torch.empty(tsu.tsu_reduce_workspace(), dtype=torch.uint8, device="cuda")
    tsu.tsu_depth_eps_gradient(g, depth, gx, gy, out, rws)
    return {"J": 0.5 * float((res.double() ** 2).sum()), "dJ_deps": float(out), "tau": sim.tau,
            "observed": obs.double().cpu().numpy()}
