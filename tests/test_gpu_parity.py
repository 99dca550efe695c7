"""GPU parity: libtsu (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: FP64 fields within 1e-12 relative L2 (the kernels evaluate the definition in the same
order without fused multiply-adds, so the observed error is round-off of the depth only);
FP32 fields within 1e-5 relative L2; integer data at Courant 1 bit for bit.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2005_11931_gb300 import inputs, tsu
from tests.gpu_helpers import relerr, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

DEPTHS = {
    "line_gauss": dict(background=1.0, eps=0.02, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5)]),
    "point_gauss": dict(background=0.5, eps=0.01, mollifier=0, sings=[(2, 1, 0.01, 0.47, 0.52)]),
    "cross_friedrichs": dict(background=1.0, eps=0.03, mollifier=1, sings=[(0, 1, 1.0, 0.5, 0.5),
                                                                          (1, 1, 0.7, 0.5, 0.41)]),
    "delta2": dict(background=1.0, eps=0.05, mollifier=0, sings=[(1, 2, 0.002, 0.5, 0.6)]),
    "step_friedrichs": dict(background=10.0, eps=0.008, mollifier=1, sings=[(3, 1, 90.0, 0.75, 0.5)]),
    "step_gauss_y": dict(background=2.0, eps=0.02, mollifier=0, sings=[(4, 1, 3.0, 0.5, 0.33)]),
    "line_point": dict(background=1.0, eps=0.015, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5), (2, 1, 0.01, 0.5, 0.5)]),
}


@pytest.mark.parametrize("name", sorted(DEPTHS))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_make_depth_matches_oracle(name, dtype):
    n, ny = 301, 257
    depth = DEPTHS[name]
    g = tsu.grid(n, ny)
    hx = tsu.empty_field(g, dtype)
    hy = tsu.empty_field(g, dtype)
    ext_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    ext = tsu.tsu_make_depth(g, depth, dtype, hx, hy, ext_dev)
    og = oracle.grid(n, ny)
    ohx, ohy, oext = oracle.make_depth(og, depth)
    ghx, ghy = hx[:, :n].double().cpu().numpy(), hy[:, :n].double().cpu().numpy()
    # FP64: the bump exp(1/(t^2-1)) amplifies rounding near its support edge (~1e-14 observed)
    tol = 1e-13 if dtype == "f64" else 1.2e-7
    if name == "step_friedrichs":
        tol = max(tol, 1e-12)
    for a, b in ((ghx, ohx), (ghy, ohy)):
        assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) <= tol
    assert np.all(hx[:, n:].cpu().numpy() == 0) and np.all(hy[:, n:].cpu().numpy() == 0)
    assert np.all(hx[:, n - 1].cpu().numpy() == 0) and np.all(hy[ny - 1, :].cpu().numpy() == 0)
    assert np.allclose(ext, oext, rtol=tol, atol=0)
    assert np.array_equal(ext, ext_dev.cpu().numpy())


def test_make_depth_rejects_nonpositive_depth():
    g = tsu.grid(64)
    hx, hy = tsu.empty_field(g, "f32"), tsu.empty_field(g, "f32")
    ext_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_make_depth(g, dict(background=0.1, eps=0.05, sings=[(2, 1, -0.01, 0.5, 0.5)]), "f32", hx, hy, ext_dev)
    assert ei.value.code == tsu.TSU_ENONPOS


def test_line_fp64_201_full_parity():
    """The 201^2 FP64 line case at its full 1000 steps: final field and the energy of every step."""
    p = inputs.line_fp64_201()
    u0 = p.initial()
    gpu = run_gpu(p.n, p.depth, u0, p.steps, dtype="f64")
    orc = run_oracle(p.n, p.depth, u0, p.steps)
    assert abs(gpu["tau"] / orc["tau"] - 1) < 1e-15
    assert relerr(gpu["u"], orc["u"]) <= 1e-12
    assert relerr(gpu["u_prev"], orc["u_prev"]) <= 1e-12
    e_g, e_o = gpu["energy"], orc["energy"]
    assert np.max(np.abs(e_g - e_o) / e_o) <= 1e-12
    # the leapfrog energy (CL-01 analogue) is conserved by the GPU run as well
    assert np.max(np.abs(e_g - e_g[0])) / e_g[0] <= 1e-12
    # the wave has reached the line: a reflection exists, the field is far from trivial
    assert np.abs(gpu["u"]).max() > 0.05


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_paper_case1_workload(dtype, tol):
    """The paper's own 2D workload (Sec. 3.3): a Friedrichs-mollified depth step from 100 to 10 at
    x = 75 (here 0.75) and the hump 50 exp(-((x-40)^2 + (y-50)^2)/8), on the unit box; 513^2
    nodes, 600 steps (the wave crosses the step and part of it is reflected)."""
    case = inputs.paper_case1_2d(n=513, steps=600)
    p = case["problem"]
    u0 = p.initial()
    gpu = run_gpu(p.n, p.depth, u0, p.steps, dtype=dtype, form=tsu.TSU_FORM_INCREMENT)
    orc = run_oracle(p.n, p.depth, u0, p.steps)
    assert relerr(gpu["u"], orc["u"]) <= tol
    assert np.max(np.abs(gpu["energy"] - orc["energy"]) / orc["energy"]) <= (1e-12 if dtype == "f64" else 1e-6)
    # the hump (width 0.028 at x = 0.40) has spread: the field left of the step is no longer the
    # initial one, and something has passed the step at x = 0.75
    assert np.abs(gpu["u"][:, int(0.8 * (p.n - 1)):]).max() > 1e-3 * 50


@pytest.mark.parametrize("form,dtype,steps,tol", [
    (tsu.TSU_FORM_STANDARD, "f64", 300, 1e-12), (tsu.TSU_FORM_INCREMENT, "f64", 300, 1e-12),
    (tsu.TSU_FORM_INCREMENT, "f32", 400, 1e-5),
    # The standard form recomputes the velocity u^n - u^{n-1} from two rounded FP32 levels every
    # step, so its round-off grows like n^1.5 ulp in the slow modes (2.9e-5 observed here); FP32
    # runs therefore default to the increment form, which meets 1e-5.
    (tsu.TSU_FORM_STANDARD, "f32", 400, 1e-4),
])
def test_ragged_grid_parity(form, dtype, steps, tol):
    """A grid that spans several CTAs in x and y with ragged tails (nx = 1000 in ld = 1024,
    ny = 777), line + point depth, Gaussian hump."""
    nx, ny = 1000, 777
    depth = DEPTHS["line_point"]
    u0 = inputs.gaussian_hump(nx, ny, None, 0.45, 0.55, 0.03)
    gpu = run_gpu(nx, depth, u0, steps, dtype=dtype, form=form, ny=ny)
    orc = run_oracle(nx, depth, u0, steps, ny=ny)
    assert relerr(gpu["u"], orc["u"]) <= tol
    assert np.max(np.abs(gpu["energy"] - orc["energy"]) / orc["energy"]) <= (1e-12 if dtype == "f64" else tol)


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 3), (3, 9), (5, 6), (130, 4), (4, 131), (513, 7)])
def test_minimal_and_thin_grids(nx, ny):
    depth = dict(background=1.0, eps=0.2, sings=[(2, 1, 0.05, 0.4, 0.6)])
    rng = np.random.default_rng(nx * 1000 + ny)
    u0 = inputs.random_field(nx, ny, None, rng)
    gpu = run_gpu(nx, depth, u0, 50, dtype="f64", ny=ny)
    orc = run_oracle(nx, depth, u0, 50, ny=ny)
    assert relerr(gpu["u"], orc["u"]) <= 1e-12
    assert np.max(np.abs(gpu["energy"] - orc["energy"]) / orc["energy"]) <= 1e-12


@pytest.mark.parametrize("S", [1, 2, 45, 256])
@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
def test_dalembert_fp32_bit_exact(S, form):
    """hx = 1, hy = 0, tau = dx = 2^-9: the FP32 kernels reproduce d'Alembert's formula with odd
    reflection exactly on even-integer data."""
    nx, ny = 513, 20
    g = tsu.grid(nx, ny)
    hx = tsu.empty_field(g, "f32")
    hy = tsu.empty_field(g, "f32")
    hx[:, : nx - 1] = 1.0
    tau = g.dx
    med = tsu.Medium(hx.data_ptr(), hy.data_ptr(), 1.0, 0.0, 1.0, 0.0)
    rng = np.random.default_rng(7)
    u0n = np.zeros((ny, nx))
    u0n[1:-1, 1:-1] = 2.0 * rng.integers(-500, 500, size=(ny - 2, nx - 2))
    u0 = tsu.empty_field(g, "f32")
    u0[:, :nx] = torch.from_numpy(u0n).float()
    bufs = [tsu.empty_field(g, "f32") for _ in range(3)]
    st = tsu.State()
    for k in range(3):
        st.buf[k] = bufs[k].data_ptr()
    st.nbuf = 3
    st.form = form
    tsu.tsu_init(g, "f32", tau, med, u0, None, st)
    tsu.tsu_step_n(g, "f32", tau, med, st, S - 1)
    u = bufs[st.cur][:, :nx].double().cpu().numpy()
    for j in range(1, ny - 1):
        F = np.concatenate([u0n[j], -u0n[j][-2:0:-1]])
        idx = np.arange(nx)
        exact = 0.5 * (F[(idx - S) % len(F)] + F[(idx + S) % len(F)])
        assert np.array_equal(u[j], exact), j


def test_separable_mode_fp64():
    nx, ny, k, l, h0, S = 129, 97, 3, 2, 1.7, 600
    depth = dict(background=h0, eps=0.1, sings=[])
    phi = inputs.separable_mode(nx, ny, None, k, l)
    gpu = run_gpu(nx, depth, phi, S, dtype="f64", ny=ny)
    g = oracle.grid(nx, ny)
    tau = gpu["tau"]
    lam = 4 * h0 / g.dx ** 2 * math.sin(k * math.pi * g.dx / 2) ** 2 + 4 * h0 / g.dy ** 2 * math.sin(
        l * math.pi * g.dy / 2) ** 2
    theta = math.acos(1 - tau * tau * lam / 2)
    assert np.max(np.abs(gpu["u"] - math.cos(S * theta) * phi)) < 1e-11


@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
def test_split_runs_are_bitwise_equal(form):
    """step_n(a) then step_n(b) equals step_n(a + b) bit for bit: the forward has no atomics, and
    the four-step passes and the single steps that finish a call round identically, so where
    the single steps fall does not matter."""
    n = 700
    depth = DEPTHS["point_gauss"]
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, tsu.grid(n).ld, 0.4, 0.5, 0.05)).float().cuda()
    sims = []
    for split in ((37, 0), (20, 17), (1, 36)):
        sim = tsu.Simulation.create(n, depth, dtype="f32", form=form)
        sim.init(u0)
        for s in split:
            if s:
                sim.step(s)
        sims.append(sim)
    torch.cuda.synchronize()
    for s in sims[1:]:
        assert torch.equal(s.u, sims[0].u)
        if form == tsu.TSU_FORM_STANDARD:
            assert torch.equal(s.u_prev, sims[0].u_prev)
        else:
            assert torch.equal(s.v, sims[0].v)


@pytest.mark.parametrize("rows", [1, 7, 32, 200])
def test_tiling_does_not_change_results(rows):
    n = 600
    depth = DEPTHS["line_gauss"]
    u0 = inputs.gaussian_hump(n, n, None, 0.3, 0.5, 0.05)
    a = run_gpu(n, depth, u0, 60, dtype="f64", rows=rows)
    b = run_oracle(n, depth, u0, 60)
    assert relerr(a["u"], b["u"]) <= 1e-12
    assert np.max(np.abs(a["energy"] - b["energy"]) / b["energy"]) <= 1e-12


def test_receiver_traces_match_oracle():
    n = 257
    rng = np.random.default_rng(inputs.SEED)
    rec = inputs.receivers_on_row(n, 0.8, 16, rng)
    rec = np.concatenate([rec, np.array([[5, 0], [n - 1, 100]])])  # two boundary receivers
    depth = DEPTHS["line_gauss"]
    u0 = inputs.gaussian_hump(n, n, None, 0.42, 0.7, 0.03)
    gpu = run_gpu(n, depth, u0, 200, dtype="f64", rec_ij=rec)
    orc = run_oracle(n, depth, u0, 200, rec_ij=rec)
    assert np.max(np.abs(gpu["traces"] - orc["traces"])) <= 1e-12 * np.abs(orc["traces"]).max()
    assert np.all(gpu["traces"][:, -2:] == 0)


@pytest.mark.parametrize("form", [tsu.TSU_FORM_STANDARD, tsu.TSU_FORM_INCREMENT])
def test_checkpoints_hold_the_state(form):
    n, S, every = 300, 50, 8
    depth = DEPTHS["line_gauss"]
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, tsu.grid(n).ld, 0.3, 0.5, 0.05)).float().cuda()
    sim = tsu.Simulation.create(n, depth, dtype="f32", form=form)
    slots = (S - 1 + every - 1) // every
    ck = torch.full((slots, 2, sim.g.ny, sim.g.ld), 7.0, dtype=torch.float32, device="cuda")
    sim.init(u0)
    sim.step(S - 1, ckpt=ck, ckpt_every=every)
    ref = tsu.Simulation.create(n, depth, dtype="f32", form=form)
    ref.init(u0)
    for c in range(slots):
        # state at step m = 1 + c*every
        if c > 0:
            ref.step(every)
        want = (ref.u_prev, ref.u) if form == tsu.TSU_FORM_STANDARD else (ref.u, ref.v)
        assert torch.equal(ck[c, 0], want[0]) and torch.equal(ck[c, 1], want[1]), c


def test_deterministic_energy():
    n = 900
    depth = DEPTHS["cross_friedrichs"]
    u0 = inputs.gaussian_hump(n, n, None, 0.3, 0.3, 0.04)
    a = run_gpu(n, depth, u0, 30, dtype="f32")
    b = run_gpu(n, depth, u0, 30, dtype="f32")
    assert np.array_equal(a["energy"], b["energy"]) and np.array_equal(a["u"], b["u"])


def test_argument_errors():
    g = tsu.grid(64)
    sim = tsu.Simulation.create(64, DEPTHS["line_gauss"], dtype="f32")
    u0 = tsu.empty_field(g, "f32")
    sim.init(u0)
    # CFL violation
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_step_n(sim.g, "f32", sim.tau * 3, sim.medium, sim.state, 1)
    assert ei.value.code == tsu.TSU_ECFL
    # ld not a multiple of 4
    bad = tsu.Grid(64, 64, 66, 1 / 63, 1 / 63)
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_step_n(bad, "f32", sim.tau, sim.medium, sim.state, 1)
    assert ei.value.code == tsu.TSU_EINVAL
    # misaligned field
    st = tsu.State()
    st.buf[0] = sim.bufs[0].data_ptr() + 4
    st.buf[1] = sim.bufs[1].data_ptr()
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_step_n(sim.g, "f32", sim.tau, sim.medium, st, 1)
    assert ei.value.code == tsu.TSU_EINVAL
    # workspace too small for the energy
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    o = tsu.StepOpts()
    o.energy = e.data_ptr()
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_step_n(sim.g, "f32", sim.tau, sim.medium, sim.state, 1, o, sim.ws, 64)
    assert ei.value.code == tsu.TSU_ENOMEM
    # nsteps = 0 is a no-op
    before = sim.u.clone()
    tsu.tsu_step_n(sim.g, "f32", sim.tau, sim.medium, sim.state, 0)
    assert torch.equal(before, sim.u)


def test_init_refuses_a_depth_that_is_not_positive():
    """A depth that dips below zero (background 0.2 minus a line of amplitude 1 at eps = 0.05, so
    min h ~ 0.2 - 11.3 < 0) breaks the positivity of Sec. 2: tsu_make_depth reports it when asked
    for the extrema on the host, and tsu_init refuses a medium built from those extrema with
    TSU_ENONPOS before it enqueues anything (the state buffers keep their contents)."""
    n = 129
    depth = dict(background=0.2, eps=0.05, mollifier=0, sings=[(0, 1, -1.0, 0.5, 0.5)])
    g = tsu.grid(n)
    hx, hy = tsu.empty_field(g, "f32"), tsu.empty_field(g, "f32")
    ext_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_make_depth(g, depth, "f32", hx, hy, ext_dev, sync=True)
    assert ei.value.code == tsu.TSU_ENONPOS
    tsu.tsu_make_depth(g, depth, "f32", hx, hy, ext_dev, sync=False)
    ext = ext_dev.cpu().numpy()
    assert ext[0] < 0 and ext[2] < 0  # h varies in x, so both face families sample the dip
    med = tsu.medium(hx, hy, ext)
    bufs = [torch.full((g.ny, g.ld), 7.0, device="cuda") for _ in range(3)]
    st = tsu.State()
    for k in range(3):
        st.buf[k] = bufs[k].data_ptr()
    st.nbuf, st.form = 3, tsu.TSU_FORM_INCREMENT
    u0 = tsu.empty_field(g, "f32")
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_init(g, "f32", 1e-4, med, u0, None, st)
    assert ei.value.code == tsu.TSU_ENONPOS
    torch.cuda.synchronize()
    assert all(bool((b == 7.0).all()) for b in bufs)
