"""GPU tests of the temporally blocked pass (several leapfrog steps per HBM pass).

It must give the scheme's result: bit for bit on integer data at Courant 1 (where FP32 is
exact), within the FP32 bars against the FP64 oracle otherwise, across strip and chunk borders,
ragged tails, tiny grids and leftover steps; and its bounded waits must report, not hang.
"""
import numpy as np
import pytest
import torch

from paper_2005_11931_gb300 import inputs, tsu
from tests.gpu_helpers import relerr, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def odd_ext_shift(f, s):
    F = np.concatenate([f, -f[-2:0:-1]])
    idx = np.arange(len(f))
    return 0.5 * (F[(idx - s) % len(F)] + F[(idx + s) % len(F)])


# (kernel, steps per pass): CTA-blocked (3) and warp-blocked (2)
BLOCKED = [(3, 4), (3, 8), (2, 2), (2, 4)]


def courant_one(axis, n_along, n_across, S, K, form, rows=64, kernel=3):
    """hx = 1, hy = 0 (axis 'x') or hx = 0, hy = 1 (axis 'y'), tau = spacing: d'Alembert exactly."""
    nx, ny = (n_along, n_across) if axis == "x" else (n_across, n_along)
    g = tsu.grid(nx, ny)
    hx = tsu.empty_field(g, "f32")
    hy = tsu.empty_field(g, "f32")
    if axis == "x":
        hx[:, : nx - 1] = 1.0
        tau, med = g.dx, None
    else:
        hy[: ny - 1, :nx] = 1.0
        tau = g.dy
    one = 1.0 if axis == "x" else 0.0  # the other face family is identically zero (a 1D problem)
    med = tsu.Medium(hx.data_ptr(), hy.data_ptr(), one, 1.0 - one, one, 1.0 - one)
    rng = np.random.default_rng(17)
    u0n = np.zeros((ny, nx))
    u0n[1:-1, 1:-1] = 2.0 * rng.integers(-300, 300, size=(ny - 2, nx - 2))
    u0 = tsu.empty_field(g, "f32")
    u0[:, :nx] = torch.from_numpy(u0n).float()
    bufs = [tsu.empty_field(g, "f32") for _ in range(4)]
    st = tsu.State()
    for k in range(4):
        st.buf[k] = bufs[k].data_ptr()
    st.nbuf, st.form = 4, form
    ws_b = tsu.tsu_step_workspace(g, "f32")
    ws = torch.zeros(ws_b, dtype=torch.uint8, device="cuda")
    tsu.tsu_init(g, "f32", tau, med, u0, None, st)
    o = tsu.StepOpts()
    o.kernel, o.tdepth, o.rows = kernel, K, rows
    tsu.tsu_step_n(g, "f32", tau, med, st, S - 1, o, ws, ws_b)
    tsu.tsu_sync_status(ws, ws_b)
    u = bufs[st.cur][:, :nx].double().cpu().numpy()
    if axis == "x":
        exact = np.stack([odd_ext_shift(u0n[j], S) for j in range(ny)])
    else:
        exact = np.stack([odd_ext_shift(u0n[:, i], S) for i in range(nx)], axis=1)
    return u, exact


@pytest.mark.parametrize("kernel,K", BLOCKED)
@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_tb_courant_one_bit_exact(kernel, K, form, axis):
    S = 1 + 5 * K + 3  # several blocked passes plus leftover single steps
    u, exact = courant_one(axis, 769, 37, S, K, form, rows=64 if kernel == 3 else 16, kernel=kernel)
    assert np.array_equal(u, exact)


@pytest.mark.parametrize("kernel,K", BLOCKED)
@pytest.mark.parametrize("form,tol", [(tsu.TSU_FORM_INCREMENT, 1e-5), (tsu.TSU_FORM_STANDARD, 1e-4)])
def test_tb_ragged_parity_with_energy(kernel, K, form, tol):
    nx, ny = 700, 613  # 3 strips (last one partial), 5 chunks of 128 rows (last one partial)
    depth = dict(background=1.0, eps=0.015, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5), (2, 1, 0.01, 0.52, 0.47)])
    u0 = inputs.gaussian_hump(nx, ny, None, 0.45, 0.55, 0.03)
    S = 1 + 12 * K + 5
    gpu = run_gpu(nx, depth, u0, S, dtype="f32", form=form, ny=ny, kernel=kernel, rows=128, tdepth=K)
    orc = run_oracle(nx, depth, u0, S, ny=ny)
    tsu.tsu_sync_status(gpu["sim"].ws, gpu["sim"].ws.numel())
    assert relerr(gpu["u"], orc["u"]) <= tol
    assert np.max(np.abs(gpu["energy"] - orc["energy"]) / orc["energy"]) <= tol


@pytest.mark.parametrize("kernel,K", [(3, 8), (2, 4), (2, 2)])
@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 4), (9, 300), (300, 6), (37, 41), (250, 251)])
def test_tb_tiny_and_thin_grids(nx, ny, kernel, K):
    depth = dict(background=1.0, eps=0.2, sings=[(2, 1, 0.05, 0.4, 0.6)])
    rng = np.random.default_rng(nx * 7 + ny)
    u0 = inputs.random_field(nx, ny, None, rng)
    S = 1 + 3 * K + 2
    gpu = run_gpu(nx, depth, u0, S, dtype="f32", ny=ny, kernel=kernel, rows=16, tdepth=K)
    orc = run_oracle(nx, depth, u0, S, ny=ny)
    assert relerr(gpu["u"], orc["u"]) <= 1e-5


@pytest.mark.parametrize("kernel,K", BLOCKED)
@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
def test_tb_matches_register_streaming_pass_bitwise(kernel, K, form):
    """Every pass rounds the same operations in the same order, so the states are equal bit for
    bit whatever the pass, depth or tiling; the energy sums differ only in summation order."""
    n = 1500
    depth = dict(background=0.5, eps=0.004, mollifier=0, sings=[(2, 1, 0.01, 0.5, 0.5)])
    u0 = inputs.gaussian_hump(n, n, None, 0.3, 0.5, 0.02)
    a = run_gpu(n, depth, u0, 201, dtype="f32", form=form, kernel=kernel, tdepth=K)
    b = run_gpu(n, depth, u0, 201, dtype="f32", form=form, kernel=1)
    assert np.array_equal(a["u"], b["u"])
    pa, pb = (a["sim"].u_prev, b["sim"].u_prev) if form == tsu.TSU_FORM_STANDARD else (a["sim"].v, b["sim"].v)
    assert torch.equal(pa, pb)
    assert np.max(np.abs(a["energy"] - b["energy"]) / b["energy"]) <= 1e-6


def test_tb_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: the test hook withholds one row copy, the consumers'
    bounded wait expires, the status word says TSU_ETIMEOUT, and the next call works."""
    n = 600
    depth = dict(background=1.0, eps=0.02, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5)])
    sim = tsu.Simulation.create(n, depth, dtype="f32")
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, sim.g.ld, 0.3, 0.5, 0.05)).float().cuda()
    sim.init(u0)
    sim.step(8, kernel=3, tdepth=8, debug=1)
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_sync_status(sim.ws, sim.ws.numel())
    assert ei.value.code == tsu.TSU_ETIMEOUT
    # the status was cleared and the context is usable
    sim2 = tsu.Simulation.create(n, depth, dtype="f32")
    sim2.init(u0)
    sim2.step(16, kernel=3, tdepth=8)
    tsu.tsu_sync_status(sim2.ws, sim2.ws.numel())
    ref = run_gpu(n, depth, u0.cpu().numpy(), 17, dtype="f32", kernel=1)
    assert relerr(sim2.u[:, :n].double().cpu().numpy(), ref["u"]) <= 1e-5


def _trace_run(kernel, n=1001, ny=777, S=61, every=8, rec=None, energy=True, form=tsu.TSU_FORM_INCREMENT,
               extra_idx=()):
    depth = dict(background=1.0, eps=0.015, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5), (2, 1, 0.01, 0.5, 0.5)])
    sim = tsu.Simulation.create(n, depth, dtype="f32", form=form, ny=ny)
    u0 = torch.from_numpy(inputs.gaussian_hump(n, ny, sim.g.ld, 0.45, 0.55, 0.03, 1.0, np.float32)).cuda()
    sim.init(u0)
    flat = np.concatenate([inputs.flat_index(rec, sim.g.ld), np.array(extra_idx, dtype=np.int64)])
    idx = torch.from_numpy(flat).cuda()
    tr = torch.full((S - 1, len(flat)), 7.0, dtype=torch.float32, device="cuda")  # every entry gets written
    ck = torch.zeros((tsu.tsu_ckpt_slots(S, every), 2, sim.g.ny, sim.g.ld), dtype=torch.float32, device="cuda")
    e = torch.zeros(S - 1, dtype=torch.float64, device="cuda") if energy else None
    sim.step(S - 1, energy=e, rec_idx=idx, traces=tr, ckpt=ck, ckpt_every=every, kernel=kernel, tdepth=4)
    torch.cuda.synchronize()
    return sim, tr, ck, e


@pytest.mark.parametrize("form", [tsu.TSU_FORM_INCREMENT, tsu.TSU_FORM_STANDARD])
@pytest.mark.parametrize("energy", [True, False])
def test_wtb_records_traces_and_checkpoints_like_one_step_passes(form, energy):
    """Receivers on and next to strip edges (columns 3/4, 115/116, 235/236; and 119/120/121,
    239/240), chunk edges, the
    corners, duplicates and boundary nodes; checkpoints every 8 steps.  The warp-blocked pass
    records them itself and copies checkpoints between launches: traces, checkpoints and states
    equal the one-step passes' bit for bit."""
    rng = np.random.default_rng(12)
    rec = [[c, r] for c in (1, 2, 3, 4, 115, 116, 119, 120, 121, 235, 236, 239, 240, 998)
           for r in (1, 2, 96, 97, 160, 161, 500, 775)]
    rec += [[120, 97], [0, 300], [500, 0], [999, 776]] + [[int(x), int(y)] for x, y in zip(
        rng.integers(1, 999, 60), rng.integers(1, 775, 60))]
    rec = np.array(rec)
    far = (-5, 10**12)  # receivers outside the grid record 0
    a, tra, cka, ea = _trace_run(2, rec=rec, energy=energy, form=form, extra_idx=far)
    b, trb, ckb, eb = _trace_run(1, rec=rec, energy=energy, form=form, extra_idx=far)
    assert not (tra == 7.0).any()
    assert torch.equal(tra, trb)
    assert torch.equal(cka, ckb)
    assert torch.equal(a.u, b.u)
    if energy:
        assert np.max(np.abs(ea.cpu().numpy() - eb.cpu().numpy()) / np.abs(eb.cpu().numpy())) <= 1e-6


def test_unaligned_checkpoints_fall_back_or_are_refused():
    rec = np.array([[10, 10], [500, 300]])
    depth = dict(background=1.0, eps=0.02, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5)])
    sim = tsu.Simulation.create(301, depth, dtype="f32")
    sim.init(torch.from_numpy(inputs.gaussian_hump(301, 301, sim.g.ld, 0.4, 0.5, 0.05, 1.0, np.float32)).cuda())
    ck = torch.zeros((8, 2, sim.g.ny, sim.g.ld), dtype=torch.float32, device="cuda")
    with pytest.raises(tsu.TsuError) as e:  # every 6 is not a multiple of 4
        sim.step(20, ckpt=ck, ckpt_every=6, kernel=2, tdepth=4)
    assert e.value.code == tsu.TSU_EINVAL
    ref = sim.clone()
    sim.step(20, ckpt=ck, ckpt_every=6)  # automatic choice: one step per pass
    ck2 = torch.zeros_like(ck)
    ref.step(20, ckpt=ck2, ckpt_every=6, kernel=1)
    torch.cuda.synchronize()
    assert torch.equal(ck, ck2) and torch.equal(sim.u, ref.u)


def test_long_receiver_lists_go_one_step_per_pass():
    """More receivers than the blocked pass scans (2048) take the one-step passes automatically."""
    rng = np.random.default_rng(21)
    rec = np.stack([rng.integers(0, 1001, 3000), rng.integers(0, 777, 3000)], axis=1)
    a, tra, cka, _ = _trace_run(0, rec=rec, energy=False)
    b, trb, ckb, _ = _trace_run(1, rec=rec, energy=False)
    assert torch.equal(tra, trb) and torch.equal(cka, ckb) and torch.equal(a.u, b.u)


def test_wtb_tile_with_more_than_32_receivers():
    """A dense 15 x 15 block of receivers (225 in one tile, more than one per lane) and duplicates
    of some of them: the warp-blocked pass reads them from its receiver table at every record;
    traces, checkpoints and states equal the one-step passes' bit for bit."""
    block = [[c, r] for c in range(40, 55) for r in range(60, 75)]
    rec = np.array(block + block[:20] + [[500, 300], [0, 5]])
    a, tra, cka, _ = _trace_run(2, rec=rec, energy=True)
    b, trb, ckb, _ = _trace_run(1, rec=rec, energy=True)
    assert not (tra == 7.0).any()
    assert torch.equal(tra, trb) and torch.equal(cka, ckb) and torch.equal(a.u, b.u)
