"""Parity at the full workload sizes, in the launch configuration bench.py times (warp-blocked
pass, 4 steps per pass, automatic rows per chunk, increment form).

The oracle cannot step 8192^2 or 16384^2 nodes for thousands of steps inside a test, so these
check
- sampled outputs: a block of nodes around the initial hump after S steps against the oracle run
  on a window of the grid whose edge lies S + 2 nodes beyond the block (the scheme moves
  information one node per step, the Taylor start included, so the window's zero edge cannot
  reach the block).  The window's depth is the same mollified depth with the singularity centres
  shifted by the window origin.  Because the waves move only a few cells in these runs, the
  change u^S - u^0 and the last increment v^S are compared too, each relative to its own size;
- properties that hold at any size: energy conservation over the whole 5000-step run and the
  x <-> y symmetry of the crossing-lines case;
- the adjoint workload at full size (2048^2, 4000 steps, 128 receivers): directional derivatives
  of the FP32 adjoint along 16 seeded random directions against central differences of the FP64
  forward (whose parity with the oracle the other tests establish).
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2005_11931_gb300 import inputs, tsu
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu


def bench_run(p, S, energy=None):
    """The bench's launch configuration: FP32 increment form, warp-blocked pass, 4 steps per pass."""
    sim = tsu.Simulation.create(p.n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    u0 = p.initial(sim.g.ld, np.float32)
    sim.init(torch.from_numpy(u0).cuda())
    sim.step(S - 1, energy=energy, kernel=2, tdepth=4)
    torch.cuda.synchronize()
    return sim, u0


def window_oracle(p, tau, u0_full, S, ic, jc, half):
    """Oracle on the window around the block [jc-half, jc+half) x [ic-half, ic+half)."""
    m = half + S + 2
    i0, j0, nw = ic - m, jc - m, 2 * m
    assert i0 >= 0 and j0 >= 0 and i0 + nw <= p.n and j0 + nw <= p.n
    og = oracle.grid(nw, nw)
    og.dx = og.dy = p.dx
    depth = dict(p.depth)
    depth["sings"] = [(k, pw, a, cx - i0 * p.dx, cy - j0 * p.dx) for (k, pw, a, cx, cy) in p.depth["sings"]]
    hx, hy, _ = oracle.make_depth(og, depth)
    u0w = np.ascontiguousarray(u0_full[j0:j0 + nw, i0:i0 + nw], dtype=np.float64)
    r = oracle.forward(og, tau, hx, hy, u0w, None, S, want_energy=False)
    blk = (slice(m - half, m + half), slice(m - half, m + half))
    return r["u"][blk], r["u"][blk] - r["u_prev"][blk], u0w[blk]


def check_block(sim, u0_full, p, S, ic, jc, half):
    ou, ov, ou0 = window_oracle(p, sim.tau, u0_full, S, ic, jc, half)
    rows, cols = slice(jc - half, jc + half), slice(ic - half, ic + half)
    gu = sim.u[rows, cols].double().cpu().numpy()
    gv = sim.v[rows, cols].double().cpu().numpy()
    e_u, e_du, e_v = relerr(gu, ou), relerr(gu - ou0, ou - ou0), relerr(gv, ov)
    assert e_u <= 1e-5, e_u
    # the change over S steps is ~1e-4 of u here; FP32 rounding of u alone is ~1e-7 of u
    assert e_du <= 5e-3, e_du
    assert e_v <= 5e-3, e_v
    return e_u, e_du, e_v


def test_point_8192_block_matches_window_oracle():
    p = inputs.point_fp32()
    S = 1000
    sim, u0 = bench_run(p, S)
    check_block(sim, u0, p, S, round(0.3 * (p.n - 1)), round(0.5 * (p.n - 1)), 128)


def test_crossing_lines_16384_block_matches_window_oracle_and_is_symmetric():
    p = inputs.crossing_lines_fp32()
    S = 1000
    sim, u0 = bench_run(p, S)
    c = round(0.25 * (p.n - 1))
    check_block(sim, u0, p, S, c, c, 96)
    # depth and data are symmetric under x <-> y
    blk = sim.u[c - 300:c + 300, c - 300:c + 300].double().cpu().numpy()
    assert relerr(blk, blk.T) <= 2e-6


# ---- FP32 against FP64 after the workloads' full step counts -----------------------------------
# The oracle cannot run 8192^2 x 5000 or 16384^2 x 20000 steps inside a test, so the reference is
# the GPU FP64 path (one step per pass, standard form, FP64 inputs), whose agreement with the
# oracle to 1e-12 the parity tests establish.  The bar is 1e-5 relative L2 of the final field.
def _fp64_reference(p, S):
    ref = tsu.Simulation.create(p.n, p.depth, dtype="f64", form=tsu.TSU_FORM_STANDARD, nbuf=2)
    u0 = torch.from_numpy(p.initial(ref.g.ld, np.float64)).cuda()
    ref.init(u0)
    ref.step(S - 1, kernel=1)
    torch.cuda.synchronize()
    out = (ref.tau, ref.u.clone(), (ref.u - ref.u_prev).clone(), u0)
    del ref
    torch.cuda.empty_cache()
    return out


def _fp32_product(p, S, tau, u0):
    """The timed configuration: FP32 increment form, automatic kernel (warp-blocked, 4 steps per
    pass) and rows."""
    sim = tsu.Simulation.create(p.n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT, tau=tau)
    sim.init(u0.float())
    sim.step(S - 1)
    torch.cuda.synchronize()
    return sim


def _rel(a, b) -> float:
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_point_8192_fp32_after_5000_steps_matches_fp64():
    """8192^2 point workload, all 5000 steps: measured 4.5e-6 relative L2."""
    p = inputs.point_fp32()
    S = p.steps
    tau, u64, v64, u0 = _fp64_reference(p, S)
    sim = _fp32_product(p, S, tau, u0)
    e_u = _rel(sim.u.double(), u64)
    assert e_u <= 1e-5, e_u
    # the part of the error that is the FP32 arithmetic alone: the FP64 path started from the
    # FP32-rounded hump (rounding u0 to FP32 perturbs v^1 = B u0 / 2 by its white-noise
    # Laplacian, ~3e-3 of v here, which no scheme can undo)
    del u64, v64
    torch.cuda.empty_cache()
    ref = tsu.Simulation.create(p.n, p.depth, dtype="f64", form=tsu.TSU_FORM_STANDARD, nbuf=2, tau=tau)
    u0r = u0.float().double()
    ref.init(u0r)
    ref.step(S - 1, kernel=1)
    torch.cuda.synchronize()
    e_du = _rel(sim.u.double() - u0r, ref.u - u0r)
    e_v = _rel(sim.v.double(), ref.u - ref.u_prev)
    print(f"8192^2 x {S}: rel L2 u {e_u:.3e}, change u^S - u^0 {e_du:.3e}, v^S {e_v:.3e}")
    assert e_du <= 1e-3, e_du
    assert e_v <= 1e-2, e_v


def test_crossing_lines_16384_fp32_after_20000_steps_matches_fp64():
    """16384^2 crossing lines, all 20000 steps (the FP64 reference takes about 2.5 minutes):
    measured 5.0e-6 relative L2."""
    p = inputs.crossing_lines_fp32()
    S = p.steps
    tau, u64, v64, u0 = _fp64_reference(p, S)
    sim = _fp32_product(p, S, tau, u0)
    e_u = _rel(sim.u.double(), u64)
    e_du = _rel(sim.u.double() - u0, u64 - u0)
    print(f"16384^2 x {S}: rel L2 u {e_u:.3e}, change u^S - u^0 {e_du:.3e}")
    assert e_u <= 1e-5, e_u
    assert e_du <= 1e-5, e_du
    del sim, u64, v64, u0
    torch.cuda.empty_cache()


def test_batched_family_members_after_2000_steps_match_the_oracle():
    """The 64-problem eps-family run batched for its full 2000 steps (the timed configuration of
    the batched measurement); the first member of every grid size, 512^2 .. 2048^2, against the
    oracle run on the same problem for the same 2000 steps."""
    probs = inputs.batched_family()
    sims = []
    for pr in probs:
        sim = tsu.Simulation.create(pr.n, pr.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
        sim.init(torch.from_numpy(pr.initial(sim.g.ld, np.float32)).cuda())
        sims.append(sim)
    nsteps = [pr.steps - 1 for pr in probs]
    wsb = tsu.tsu_batch_workspace(sims, nsteps)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_batch_run(sims, nsteps, ws, wsb)
    tsu.tsu_sync_status(ws, wsb)
    first = {}
    for k, pr in enumerate(probs):
        first.setdefault(pr.n, k)
    assert sorted(first) == [512, 768, 1024, 1536, 2048]
    oracle.set_threads(len(os.sched_getaffinity(0)))
    errs = {}
    for n, k in sorted(first.items()):
        pr, sim = probs[k], sims[k]
        g = oracle.grid(n, n)
        hx, hy, _ = oracle.make_depth(g, pr.depth)
        ref = oracle.forward(g, sim.tau, hx, hy, pr.initial(), None, pr.steps, want_energy=False)
        errs[n] = relerr(sim.u[:, :n].double().cpu().numpy(), ref["u"])
    print("family members after 2000 steps, rel L2:", {n: f"{e:.2e}" for n, e in errs.items()})
    assert max(errs.values()) <= 1e-5, errs


def test_point_8192_full_run_conserves_energy():
    p = inputs.point_fp32()
    e = torch.zeros(p.steps - 1, dtype=torch.float64, device="cuda")
    bench_run(p, p.steps, energy=e)
    en = e.cpu().numpy()
    assert np.all(en > 0)
    drift = np.max(np.abs(en - en[0])) / en[0]
    # FP32 fields, FP64 sums: the leapfrog energy is exactly conserved, rounding of the states
    # alone moves it
    assert drift <= 1e-4, drift


def _forward_traces(p, depth, dtype, tau, rec_ij, hx=None, hy=None, ck=None, every=64):
    form = tsu.TSU_FORM_INCREMENT if dtype == "f32" else tsu.TSU_FORM_STANDARD
    sim = tsu.Simulation.create(p.n, depth, dtype=dtype, form=form, tau=tau)
    if hx is not None:
        sim.hx.copy_(hx)
        sim.hy.copy_(hy)
    tdt = tsu.DTYPES[sim.dtype]
    g = sim.g
    u0 = torch.from_numpy(p.initial(g.ld, np.float64)).to(tdt).cuda()
    rec = torch.from_numpy(inputs.flat_index(rec_ij, g.ld)).cuda()
    S = p.steps
    tr = torch.zeros((S, rec.numel()), dtype=tdt, device="cuda")
    sim.init(u0)
    sim.step(S - 1, rec_idx=rec, traces=tr[: S - 1], ckpt=ck, ckpt_every=every if ck is not None else 0)
    sim.observe(rec_idx=rec, trace=tr[S - 1])
    torch.cuda.synchronize()
    return sim, u0, rec, tr


def test_adjoint_2048_full_size_directional_derivatives():
    case = inputs.adjoint_case()
    p, rec_ij = case["problem"], case["receivers"]
    S, every = p.steps, case["ckpt_every"]
    ref = tsu.Simulation.create(p.n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    tau = ref.tau
    # observations from the other medium (eps = 0.012), FP64
    _, _, _, obs = _forward_traces(p, case["depth_obs"], "f64", tau, rec_ij)
    # FP32 forward with checkpoints, then the FP32 adjoint
    g = ref.g
    ck = torch.zeros((tsu.tsu_ckpt_slots(S, every), 2, g.ny, g.ld), dtype=torch.float32, device="cuda")
    sim, u0, rec, tr = _forward_traces(p, p.depth, "f32", tau, rec_ij, ck=ck, every=every)
    out = {k: torch.zeros((g.ny, g.ld), dtype=torch.float64 if k in ("gx", "gy") else torch.float32, device="cuda")
           for k in ("gx", "gy", "gu0", "gu1")}
    wsb = tsu.tsu_adjoint_workspace(g, tsu.TSU_F32, tsu.TSU_FORM_INCREMENT, S, every, rec.numel())
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_adjoint(g, tsu.TSU_F32, tsu.TSU_FORM_INCREMENT, tau, sim.medium, S, every, ck, u0, rec,
                    (tr.double() - obs).float(), out["gx"], out["gy"], out["gu0"], out["gu1"], ws, wsb)
    torch.cuda.synchronize()
    # J and its central differences with the FP64 forward
    hx64 = sim.hx.double()
    hy64 = sim.hy.double()
    mask_x = torch.zeros_like(hx64)
    mask_x[1:-1, : p.n - 1] = 1
    mask_y = torch.zeros_like(hy64)
    mask_y[: p.n - 1, 1:p.n - 1] = 1

    def J(hx, hy):
        _, _, _, t = _forward_traces(p, p.depth, "f64", tau, rec_ij, hx=hx, hy=hy)
        return 0.5 * float(((t - obs) ** 2).sum())

    gen = torch.Generator(device="cpu").manual_seed(inputs.SEED)
    for trial in range(16):  # the workload's 16 seeded random directions
        dx_ = (torch.randn(hx64.shape, generator=gen, dtype=torch.float64).cuda() * mask_x)
        dy_ = (torch.randn(hy64.shape, generator=gen, dtype=torch.float64).cuda() * mask_y)
        st = 1e-3
        fd = (J(hx64 + st * dx_, hy64 + st * dy_) - J(hx64 - st * dx_, hy64 - st * dy_)) / (2 * st)
        ad = float((out["gx"] * dx_).sum() + (out["gy"] * dy_).sum())
        assert abs(fd - ad) <= 1e-4 * abs(fd), (trial, fd, ad)


def test_grid_beyond_2_31_elements():
    """47000^2 nodes (ld 47008: 2.21e9 elements per field, past 2^31; six FP32 fields = 53 GB):
    64-bit indexing in the depth, start, blocked and single-step passes.  The input is a hump of
    compact support (zero outside a 401^2 block) so that the oracle's window stays small."""
    n, S, half = 47000, 11, 60
    p = inputs.Problem("big", n, dict(background=1.0, eps=8.0 / (n - 1), mollifier=0,
                                      sings=[(0, 1, 1.0, 0.9, 0.5), (1, 1, 1.0, 0.5, 0.9)]),
                       (0.9, 0.9, 0.0, 1.0), S)
    sim = tsu.Simulation.create(n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    assert sim.g.ny * sim.g.ld > 2**31
    # hump of width 40 dx at the node nearest (0.9, 0.9), i.e. near the far corner of the arrays
    ic = jc = round(0.9 * (n - 1))
    blk = 200
    w = 40.0 / (n - 1)
    small = inputs.gaussian_hump(2 * blk + 1, 2 * blk + 1, None, 0.5, 0.5, w * (n - 1) / (2 * blk), 1.0)
    u0 = torch.zeros((sim.g.ny, sim.g.ld), dtype=torch.float32, device="cuda")
    u0[jc - blk:jc + blk + 1, ic - blk:ic + blk + 1] = torch.from_numpy(small).float()
    sim.init(u0)
    sim.step(S - 1, kernel=2, tdepth=4)  # two blocked passes and two single steps
    torch.cuda.synchronize()
    # oracle on a window around the hump with the same input block
    m = half + S + 2
    i0, j0, nw = ic - m, jc - m, 2 * m
    og = oracle.grid(nw, nw)
    og.dx = og.dy = 1.0 / (n - 1)
    depth = dict(p.depth)
    depth["sings"] = [(k, pw, a, cx - i0 * og.dx, cy - j0 * og.dx) for (k, pw, a, cx, cy) in p.depth["sings"]]
    hx, hy, _ = oracle.make_depth(og, depth)
    u0w = u0[j0:j0 + nw, i0:i0 + nw].double().cpu().numpy()
    r = oracle.forward(og, sim.tau, hx, hy, u0w, None, S, want_energy=False)
    ref = r["u"][m - half:m + half, m - half:m + half]
    got = sim.u[jc - half:jc + half, ic - half:ic + half].double().cpu().numpy()
    assert relerr(got, ref) <= 1e-5
    # the far end of the arrays is written (zeros), the last interior row holds finite values
    assert torch.isfinite(sim.u[-2, :n]).all()
    del sim, u0
    torch.cuda.empty_cache()
