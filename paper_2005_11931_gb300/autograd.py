"""``torch.autograd.Function`` around the leapfrog forward and its discrete adjoint.

``TsunamiFn.apply(hx, hy, u0, u1, cfg)`` runs the Taylor start and ``cfg.steps - 1`` leapfrog
steps through libtsu, recording ``u^n`` at the receivers for n = 1..S (a [S, nrec] tensor) and
checkpointing the state every ``cfg.ckpt_every`` steps.  ``backward`` hands dJ/dtraces to
``tsu_adjoint``, which recomputes each checkpoint segment and runs the reverse-time adjoint, and
returns dJ/dhx, dJ/dhy (FP64 accumulated, cast to the field type), dJ/du0 and dJ/du1.
Marshalling only: all arithmetic is in the CUDA kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import tsu


@dataclass
class TsunamiConfig:
    grid: tsu.Grid
    tau: float
    steps: int                 # S: the final state is u^S (the Taylor start is step 1)
    rec_idx: torch.Tensor      # int64 flat node indices j*ld + i (device)
    ext: tuple                 # face extrema [min hx, max hx, min hy, max hy] (from tsu_make_depth)
    form: int = tsu.TSU_FORM_INCREMENT
    ckpt_every: int = 64


class TsunamiFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, hx, hy, u0, u1, cfg: TsunamiConfig):
        g, S = cfg.grid, int(cfg.steps)
        code = tsu.dtype_code(u0.dtype)
        dev = u0.device
        for t, name in ((hx, "hx"), (hy, "hy"), (u0, "u0"), (u1, "u1")):
            if t is not None and tuple(t.shape) != (g.ny, g.ld):
                raise ValueError(f"{name} must have shape (ny, ld) = {(g.ny, g.ld)} (got {tuple(t.shape)})")
        med = tsu.Medium(tsu._field(hx, g, code, "hx"), tsu._field(hy, g, code, "hy"), float(cfg.ext[1]),
                         float(cfg.ext[3]), float(cfg.ext[0]), float(cfg.ext[2]))
        # four state buffers: FP32 runs then take the warp-blocked pass (receivers and checkpoints
        # recorded by it), FP64 runs one step per pass
        bufs = [torch.zeros_like(u0) for _ in range(4)]
        st = tsu.State()
        for k, b in enumerate(bufs):
            st.buf[k] = b.data_ptr()
        st.nbuf, st.form = 4, cfg.form
        nrec = int(cfg.rec_idx.numel())
        traces = torch.zeros((S, nrec), dtype=u0.dtype, device=dev)
        slots = max(tsu.tsu_ckpt_slots(S, cfg.ckpt_every), 1)
        ckpt = torch.empty((slots, 2) + tuple(u0.shape), dtype=u0.dtype, device=dev)
        ws_b = tsu.tsu_step_workspace(g, code)
        ws = torch.zeros(ws_b, dtype=torch.uint8, device=dev)
        tsu.tsu_init(g, code, cfg.tau, med, u0, u1, st)
        if S > 1:
            o = tsu.StepOpts()
            o.nrec, o.rec_idx, o.traces = nrec, cfg.rec_idx.data_ptr(), traces.data_ptr()
            o.ckpt, o.ckpt_every, o.ckpt_slots = ckpt.data_ptr(), int(cfg.ckpt_every), slots
            tsu.tsu_step_n(g, code, cfg.tau, med, st, S - 1, o, ws, ws_b)
        tsu.tsu_observe(g, code, cfg.tau, med, st, None, cfg.rec_idx, traces[S - 1], ws, ws_b)
        ctx.save_for_backward(hx, hy, u0, ckpt)
        ctx.cfg = cfg
        return traces

    @staticmethod
    def backward(ctx, dtraces):
        hx, hy, u0, ckpt = ctx.saved_tensors
        cfg = ctx.cfg
        g, S = cfg.grid, int(cfg.steps)
        code = tsu.dtype_code(u0.dtype)
        nrec = int(cfg.rec_idx.numel())
        if tuple(dtraces.shape) != (S, nrec):
            raise ValueError(f"dtraces must have shape [S, nrec] = {(S, nrec)} (got {tuple(dtraces.shape)})")
        med = tsu.Medium(tsu._field(hx, g, code, "hx"), tsu._field(hy, g, code, "hy"), float(cfg.ext[1]),
                         float(cfg.ext[3]), float(cfg.ext[0]), float(cfg.ext[2]))
        dev = u0.device
        g_hx = torch.zeros(u0.shape, dtype=torch.float64, device=dev)
        g_hy = torch.zeros(u0.shape, dtype=torch.float64, device=dev)
        g_u0 = torch.zeros_like(u0)
        g_u1 = torch.zeros_like(u0)
        ws_b = tsu.tsu_adjoint_workspace(g, code, cfg.form, S, cfg.ckpt_every, int(cfg.rec_idx.numel()))
        ws = torch.empty(ws_b, dtype=torch.uint8, device=dev)
        tsu.tsu_adjoint(g, code, cfg.form, cfg.tau, med, S, cfg.ckpt_every, ckpt, u0, cfg.rec_idx,
                        dtraces.contiguous().to(u0.dtype), g_hx, g_hy, g_u0, g_u1, ws, ws_b)
        return g_hx.to(hx.dtype), g_hy.to(hy.dtype), g_u0, g_u1, None


def tsunami_traces(hx, hy, u0, u1, cfg: TsunamiConfig) -> torch.Tensor:
    """Receiver traces u^n(rec), n = 1..S, differentiable in hx, hy, u0 and u1."""
    if u1 is None:
        u1 = torch.zeros_like(u0)
    return TsunamiFn.apply(hx, hy, u0, u1, cfg)
