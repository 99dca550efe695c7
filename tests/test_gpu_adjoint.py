"""GPU tests of the discrete adjoint (tsu_adjoint) and the autograd wrapper.

The adjoint must equal the oracle's FP64 discrete adjoint (same recursion, same order) and the
derivative of the forward map (central differences of the oracle's forward), for both forward
forms, any checkpoint period, duplicate and boundary receivers.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2005_11931_gb300 import inputs, tsu
from paper_2005_11931_gb300.autograd import TsunamiConfig, tsunami_traces
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu

DEPTH = dict(background=1.0, eps=0.06, mollifier=0, sings=[(0, 1, 0.5, 0.5, 0.5), (2, 1, 0.002, 0.4, 0.6)])


def gpu_forward_adjoint(nx, ny, depth, u0n, u1n, S, rec_ij, dtr, dtype, form, every):
    """Forward with checkpoints through tsu_step_n, then tsu_adjoint.  Returns numpy gradients."""
    sim = tsu.Simulation.create(nx, depth, dtype=dtype, form=form, ny=ny, nbuf=3)
    g = sim.g
    tdt = tsu.DTYPES[sim.dtype]
    pad = lambda a: torch.from_numpy(np.pad(a[:, :nx], ((0, 0), (0, g.ld - nx)))).to(tdt).cuda()
    u0, u1 = pad(u0n), pad(u1n)
    sim.init(u0, u1)
    slots = max(tsu.tsu_ckpt_slots(S, every), 1)
    ck = torch.zeros((slots, 2, g.ny, g.ld), dtype=tdt, device="cuda")
    if S > 1:
        sim.step(S - 1, ckpt=ck, ckpt_every=every)
    rec = torch.from_numpy(inputs.flat_index(rec_ij, g.ld)).cuda()
    dt = torch.from_numpy(dtr).to(tdt).cuda()
    out = {k: torch.zeros((g.ny, g.ld), dtype=torch.float64 if k in ("g_hx", "g_hy") else tdt, device="cuda")
           for k in ("g_hx", "g_hy", "g_u0", "g_u1")}
    wsb = tsu.tsu_adjoint_workspace(g, sim.dtype, form, S, every, len(rec))
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_adjoint(g, sim.dtype, form, sim.tau, sim.medium, S, every, ck, u0, rec, dt, out["g_hx"], out["g_hy"],
                    out["g_u0"], out["g_u1"], ws, wsb)
    torch.cuda.synchronize()
    return {k: v[:, :nx].double().cpu().numpy() for k, v in out.items()}, sim.tau


def receivers(nx, ny):
    rng = np.random.default_rng(inputs.SEED)
    rec = inputs.receivers_on_row(nx, 0.7, 6, rng)
    # a duplicate and a boundary receiver
    return np.concatenate([rec, rec[2:3], np.array([[0, ny // 2]])])


@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
@pytest.mark.parametrize("every,S", [(1, 30), (7, 61), (64, 61), (10, 2), (5, 1)])
def test_fp64_adjoint_matches_oracle(form, every, S):
    nx, ny = 61, 47
    rng = np.random.default_rng(11)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    rec = receivers(nx, ny)
    dtr = rng.standard_normal((S, len(rec)))
    gg, tau = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f64", form, every)
    og = oracle.grid(nx, ny)
    hx, hy, ext = oracle.make_depth(og, DEPTH)
    ref = oracle.adjoint(og, tau, hx, hy, u0, u1, S, inputs.flat_index(rec, nx), dtr)
    tol = 1e-12 if form == tsu.TSU_FORM_STANDARD else 1e-10  # the increment form rounds its states differently
    for k in ("g_hx", "g_hy", "g_u0", "g_u1"):
        assert relerr(gg[k], ref[k]) <= tol, (k, relerr(gg[k], ref[k]))


def test_fp64_adjoint_independent_of_checkpoint_period():
    nx, ny, S = 90, 70, 150
    rng = np.random.default_rng(2)
    u0 = inputs.gaussian_hump(nx, ny, None, 0.4, 0.5, 0.1)
    u1 = np.zeros_like(u0)
    rec = receivers(nx, ny)
    dtr = rng.standard_normal((S, len(rec)))
    a, _ = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f64", tsu.TSU_FORM_STANDARD, 1)
    b, _ = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f64", tsu.TSU_FORM_STANDARD, 37)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
@pytest.mark.parametrize("every,S", [(8, 41), (5, 23), (64, 41), (3, 2)])
def test_fp32_adjoint_matches_oracle_across_tiles(form, every, S):
    """FP32 sweeps run four adjoint steps per pass on 120-column by 16-row tiles, with single
    passes for the rest of a segment.  Against the FP64 oracle on a grid of 3 strips and a ragged
    last chunk, with receivers on and up to three rows and four columns beyond strip and chunk
    edges (where halo copies of a multiplier need the receiver value too), duplicates and a
    boundary receiver."""
    nx, ny = 301, 150
    rng = np.random.default_rng(23)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    cols = [1, 3, 4, 111, 112, 115, 116, 119, 120, 123, 124, 231, 232, 235, 236, 239, 240, 243, 299]
    rows = [1, 2, 3, 13, 14, 15, 16, 17, 18, 19, 20, 32, 33, 144, 145, 147, 148]
    rec = np.array([[cols[k % len(cols)], rows[k % len(rows)]] for k in range(3 * len(cols))]
                   + [[120, 17], [0, 40], [150, 149]])
    dtr = rng.standard_normal((S, len(rec)))
    gg, tau = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f32", form, every)
    og = oracle.grid(nx, ny)
    hx, hy, ext = oracle.make_depth(og, DEPTH)
    ref = oracle.adjoint(og, tau, hx, hy, u0, u1, S, inputs.flat_index(rec, nx), dtr)
    for k in ("g_hx", "g_hy", "g_u0", "g_u1"):
        # FP32 states and multipliers: rounding of order 1e-7 per step, grown over S steps
        assert relerr(gg[k], ref[k]) <= 2e-5, (k, relerr(gg[k], ref[k]))
        assert np.max(np.abs(gg[k] - ref[k])) <= 1e-4 * np.max(np.abs(ref[k])), k


def test_fp32_adjoint_full_gradients_at_256_and_500_steps():
    """The adjoint workload's problem at a size the FP64 oracle adjoint takes whole (256^2, 500
    steps, 32 receivers on y = 0.8, checkpoints every 20): every gradient field (dJ/dhx, dJ/dhy,
    dJ/du0, dJ/du1) of the FP32 GPU adjoint against the oracle's FP64 one.  Measured relative L2
    errors are a few 1e-6; the bar is 2e-5."""
    case = inputs.adjoint_case(n=256, steps=500, nrec=32)
    p = case["problem"]
    n, S = p.n, p.steps
    rng = np.random.default_rng(31)
    u0 = p.initial()
    u1 = np.zeros_like(u0)
    dtr = 1e-2 * rng.standard_normal((S, len(case["receivers"])))
    gg, tau = gpu_forward_adjoint(n, n, p.depth, u0, u1, S, case["receivers"], dtr, "f32", tsu.TSU_FORM_INCREMENT,
                                  20)
    og = oracle.grid(n, n)
    hx, hy, ext = oracle.make_depth(og, p.depth)
    ref = oracle.adjoint(og, tau, hx, hy, u0, u1, S, inputs.flat_index(case["receivers"], n), dtr)
    for k in ("g_hx", "g_hy", "g_u0", "g_u1"):
        assert relerr(gg[k], ref[k]) <= 2e-5, (k, relerr(gg[k], ref[k]))


@pytest.mark.parametrize("S,every", [(69, 64), (46, 16)])
def test_fp32_adjoint_1600_matches_fp64_adjoint(S, every):
    """The FP32 adjoint on a 1600^2 grid (the four-step reverse pass over many tiles) against the
    FP64 GPU adjoint (one step per pass, itself equal to the oracle to 1e-12) on the same problem,
    with segments of 16 passes, of one pass and of leftover single steps, 24 receivers.  A wrong
    state or multiplier would show at order 1.  FP32 rounding stays near 1e-7 in dJ/du0, dJ/du1;
    the face gradients sum products of differences of u and lam over the steps and lose more
    (measured 4.5e-6 and 4.2e-5 for dJ/dhx in the two cases)."""
    n = 1600
    rng = np.random.default_rng(37)
    u0 = inputs.gaussian_hump(n, n, None, 0.45, 0.55, 0.03)
    u1 = np.zeros_like(u0)
    rec = np.stack([rng.integers(1, n - 1, 24), rng.integers(1, n - 1, 24)], axis=1)
    dtr = rng.standard_normal((S, len(rec)))
    a, _ = gpu_forward_adjoint(n, n, DEPTH, u0, u1, S, rec, dtr, "f32", tsu.TSU_FORM_INCREMENT, every)
    b, _ = gpu_forward_adjoint(n, n, DEPTH, u0, u1, S, rec, dtr, "f64", tsu.TSU_FORM_STANDARD, every)
    errs = {k: relerr(a[k], b[k]) for k in ("g_hx", "g_hy", "g_u0", "g_u1")}
    assert errs["g_u0"] <= 2e-5 and errs["g_u1"] <= 2e-5, errs
    assert errs["g_hx"] <= 1e-4 and errs["g_hy"] <= 1e-4, errs


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 6), (17, 9), (130, 5), (6, 140)])
def test_fp32_adjoint_tiny_and_thin_grids(nx, ny):
    """The four-step pass on grids smaller than a tile in one or both directions (one strip,
    one chunk, a single interior row or column), against the FP64 oracle."""
    S, every = 23, 8
    rng = np.random.default_rng(nx * 1000 + ny)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    rec = np.array([[nx // 2, ny // 2], [1, 1], [nx - 2, ny - 2], [0, ny // 2]])
    dtr = rng.standard_normal((S, len(rec)))
    gg, tau = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f32", tsu.TSU_FORM_INCREMENT, every)
    og = oracle.grid(nx, ny)
    hx, hy, ext = oracle.make_depth(og, DEPTH)
    ref = oracle.adjoint(og, tau, hx, hy, u0, u1, S, inputs.flat_index(rec, nx), dtr)
    for k in ("g_hx", "g_hy", "g_u0", "g_u1"):
        if np.abs(ref[k]).max() == 0:
            assert np.abs(gg[k]).max() == 0, k
        else:
            assert relerr(gg[k], ref[k]) <= 2e-5, (k, relerr(gg[k], ref[k]))


def test_fp32_adjoint_directional_derivatives_match_central_differences():
    """FP32 fields, FP64-accumulated face gradients: <dJ/dh, d> against central differences of the
    oracle's FP64 forward map along seeded random directions, relative error <= 1e-4."""
    n, S, every = 97, 240, 64
    depth = dict(background=1.0, eps=0.04, mollifier=0, sings=[(0, 1, 0.5, 0.5, 0.5)])
    rng = np.random.default_rng(inputs.SEED)
    u0 = inputs.gaussian_hump(n, n, None, 0.42, 0.70, 0.06)
    u1 = np.zeros_like(u0)
    rec = inputs.receivers_on_row(n, 0.8, 16, rng)
    og = oracle.grid(n, n)
    hx, hy, ext = oracle.make_depth(og, depth)
    tau = 0.4 * og.dx / math.sqrt(max(ext[1], ext[3]))
    ridx = inputs.flat_index(rec, n)
    obs = oracle.forward(og, tau, hx * 1.05, hy * 1.05, u0, None, S, want_energy=False, rec_idx=ridx)["traces"]

    def J(hx_, hy_):
        tr = oracle.forward(og, tau, hx_, hy_, u0, None, S, want_energy=False, rec_idx=ridx)["traces"]
        return 0.5 * float(np.sum((tr - obs) ** 2)), tr

    J0, tr0 = J(hx, hy)
    gg, gtau = gpu_forward_adjoint(n, n, depth, u0, u1, S, rec, tr0 - obs, "f32", tsu.TSU_FORM_INCREMENT, every)
    assert abs(gtau / tau - 1) < 1e-6
    mx = np.zeros_like(hx)
    mx[:, : n - 1] = 1
    my = np.zeros_like(hy)
    my[: n - 1, :] = 1
    for trial in range(8):
        dx_ = rng.standard_normal(hx.shape) * mx
        dy_ = rng.standard_normal(hy.shape) * my
        st = 1e-4
        fd = (J(hx + st * dx_, hy + st * dy_)[0] - J(hx - st * dx_, hy - st * dy_)[0]) / (2 * st)
        ad = float(np.sum(gg["g_hx"] * dx_) + np.sum(gg["g_hy"] * dy_))
        assert abs(fd - ad) <= 1e-4 * abs(fd), (trial, fd, ad)


def test_tsunami_fn_autograd_matches_oracle_adjoint():
    n, S = 80, 120
    depth = dict(background=1.0, eps=0.05, mollifier=0, sings=[(0, 1, 0.5, 0.5, 0.5)])
    sim = tsu.Simulation.create(n, depth, dtype="f64", form=tsu.TSU_FORM_STANDARD)
    g = sim.g
    rng = np.random.default_rng(4)
    rec = inputs.receivers_on_row(n, 0.8, 10, rng)
    u0n = inputs.gaussian_hump(n, n, g.ld, 0.45, 0.6, 0.08)
    obs = torch.from_numpy(rng.standard_normal((S, len(rec))) * 1e-3).cuda()
    hx = sim.hx.clone().requires_grad_(True)
    hy = sim.hy.clone().requires_grad_(True)
    u0 = torch.from_numpy(u0n).cuda().requires_grad_(True)
    u1 = torch.zeros_like(u0).requires_grad_(True)
    cfg = TsunamiConfig(g, sim.tau, S, torch.from_numpy(inputs.flat_index(rec, g.ld)).cuda(), tuple(sim.ext),
                        form=tsu.TSU_FORM_STANDARD, ckpt_every=16)
    tr = tsunami_traces(hx, hy, u0, u1, cfg)
    loss = 0.5 * ((tr - obs) ** 2).sum()
    loss.backward()
    og = oracle.grid(n, n)
    ohx, ohy, _ = oracle.make_depth(og, depth)
    fwd = oracle.forward(og, sim.tau, ohx, ohy, u0n[:, :n], None, S, want_energy=False,
                         rec_idx=inputs.flat_index(rec, n))
    assert relerr(tr.detach().cpu().numpy(), fwd["traces"]) <= 1e-12
    ref = oracle.adjoint(og, sim.tau, ohx, ohy, u0n[:, :n], None, S, inputs.flat_index(rec, n),
                         fwd["traces"] - obs.cpu().numpy())
    assert relerr(hx.grad[:, :n].cpu().numpy(), ref["g_hx"]) <= 1e-11
    assert relerr(hy.grad[:, :n].cpu().numpy(), ref["g_hy"]) <= 1e-11
    assert relerr(u0.grad[:, :n].cpu().numpy(), ref["g_u0"]) <= 1e-11
    assert relerr(u1.grad[:, :n].cpu().numpy(), ref["g_u1"]) <= 1e-11


def test_tsunami_fn_autograd_fp32():
    """The autograd wrapper on FP32 fields (warp-blocked forward recording receivers and
    checkpoints, four-step reverse passes): traces and gradients against the FP64 oracle."""
    n, S = 161, 130
    depth = dict(background=1.0, eps=0.05, mollifier=0, sings=[(0, 1, 0.5, 0.5, 0.5)])
    sim = tsu.Simulation.create(n, depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    g = sim.g
    rng = np.random.default_rng(14)
    rec = inputs.receivers_on_row(n, 0.8, 10, rng)
    u0n = inputs.gaussian_hump(n, n, g.ld, 0.45, 0.6, 0.08)
    obs = torch.from_numpy(rng.standard_normal((S, len(rec))) * 1e-3).float().cuda()
    hx = sim.hx.clone().requires_grad_(True)
    hy = sim.hy.clone().requires_grad_(True)
    u0 = torch.from_numpy(u0n).float().cuda().requires_grad_(True)
    u1 = torch.zeros_like(u0).requires_grad_(True)
    cfg = TsunamiConfig(g, sim.tau, S, torch.from_numpy(inputs.flat_index(rec, g.ld)).cuda(), tuple(sim.ext),
                        form=tsu.TSU_FORM_INCREMENT, ckpt_every=16)
    tr = tsunami_traces(hx, hy, u0, u1, cfg)
    loss = 0.5 * ((tr - obs) ** 2).sum()
    loss.backward()
    og = oracle.grid(n, n)
    ohx, ohy, _ = oracle.make_depth(og, depth)
    fwd = oracle.forward(og, sim.tau, ohx, ohy, u0n[:, :n], None, S, want_energy=False,
                         rec_idx=inputs.flat_index(rec, n))
    assert relerr(tr.detach().double().cpu().numpy(), fwd["traces"]) <= 1e-5
    ref = oracle.adjoint(og, sim.tau, ohx, ohy, u0n[:, :n], None, S, inputs.flat_index(rec, n),
                         tr.detach().double().cpu().numpy() - obs.double().cpu().numpy())
    assert relerr(hx.grad[:, :n].double().cpu().numpy(), ref["g_hx"]) <= 2e-5
    assert relerr(hy.grad[:, :n].double().cpu().numpy(), ref["g_hy"]) <= 2e-5
    assert relerr(u0.grad[:, :n].double().cpu().numpy(), ref["g_u0"]) <= 2e-5
    assert relerr(u1.grad[:, :n].double().cpu().numpy(), ref["g_u1"]) <= 2e-5


def test_adjoints_from_two_host_threads():
    """Two host threads enqueue adjoints on their own streams at the same time; each gets the
    result of a run alone (the recompute streams and their events are per thread)."""
    import threading

    nx, ny, S, every = 150, 120, 45, 8
    rng = np.random.default_rng(31)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    rec = receivers(nx, ny)
    dtr = rng.standard_normal((S, len(rec)))
    alone = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f32", tsu.TSU_FORM_INCREMENT, every)[0]
    out, errs = [None, None], []

    def work(k):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                for _ in range(3):
                    out[k] = gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f32",
                                                 tsu.TSU_FORM_INCREMENT, every)[0]
        except Exception as ex:  # pragma: no cover - reported below
            errs.append(ex)

    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for k in range(2):
        for name in alone:
            assert np.array_equal(out[k][name], alone[name]), (k, name)


def test_adjoint_streams_released_when_threads_exit():
    """tsu_adjoint creates one auxiliary stream (and its events) per calling host thread; they are
    destroyed when that thread exits, so adjoints run from many short-lived threads do not
    accumulate streams."""
    import threading
    import time

    nx, ny, S, every = 97, 80, 21, 8
    rng = np.random.default_rng(41)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    rec = receivers(nx, ny)
    dtr = rng.standard_normal((S, len(rec)))
    gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f32", tsu.TSU_FORM_INCREMENT, every)

    def stable():
        # threads of earlier tests may still be running their thread-local destructors: take the
        # count once it has not changed for half a second
        deadline = time.monotonic() + 10.0
        last, since = tsu.tsu_aux_streams(), time.monotonic()
        while time.monotonic() < deadline:
            time.sleep(0.01)
            v = tsu.tsu_aux_streams()
            if v != last:
                last, since = v, time.monotonic()
            elif time.monotonic() - since > 0.5:
                break
        return last

    base = stable()
    assert base >= 1  # this thread's stream
    seen, errs = [], []

    def work():
        try:
            torch.cuda.set_device(0)
            gpu_forward_adjoint(nx, ny, DEPTH, u0, u1, S, rec, dtr, "f32", tsu.TSU_FORM_INCREMENT, every)
            seen.append(tsu.tsu_aux_streams())
        except Exception as ex:  # pragma: no cover - reported below
            errs.append(ex)

    def settled():
        # Thread.join() returns once the thread's Python part is done; the OS thread runs its C++
        # thread-local destructors (which release the stream) a moment later
        deadline = time.monotonic() + 10.0
        while tsu.tsu_aux_streams() != base and time.monotonic() < deadline:
            time.sleep(0.005)
        return tsu.tsu_aux_streams()

    for _ in range(6):
        t = threading.Thread(target=work)
        t.start()
        t.join()
        assert settled() == base
    assert not errs, errs
    assert seen == [base + 1] * 6, (base, seen)  # the running thread's own, while it lives
