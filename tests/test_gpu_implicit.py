"""GPU parity of the implicit comparator (Sec. 3.3, read as the factorized scheme
(I - s B_x)(I - s B_y) w^n = B u^n): libtsu through the C ABI against the FP64 oracle's
line-by-line Thomas solves, on the same seeded inputs.

Bars: FP64 fields within 1e-12 relative L2, FP32 within 1e-5.  The GPU solves every line by a
warp scan of affine maps, so its rounding differs from sequential elimination; the bars hold at
time steps far beyond the explicit Courant limit.  The closed-form separable mode checks the
GPU at sizes the oracle would take long to reach.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2005_11931_gb300 import inputs, tsu
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu

DEPTHS = {
    "line_point": dict(background=1.0, eps=0.03, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5), (2, 1, 0.01, 0.45, 0.55)]),
    "cross_friedrichs": dict(background=1.0, eps=0.04, mollifier=1, sings=[(0, 1, 1.0, 0.5, 0.5),
                                                                          (1, 1, 0.7, 0.5, 0.41)]),
    "paper_step": dict(background=10.0, eps=0.008, mollifier=1, sings=[(3, 1, 90.0, 0.75, 0.5)]),
}


def run_pair(nx, ny, depth, S, dtype, cfl=None, tau=None, sigma=0.25, with_u1=True, u0_spec=(0.4, 0.45, 0.1, 1.0),
             seed=3):
    """The GPU implicit run and the oracle's on the same inputs (tau from the Courant number
    when not given); returns (gpu u, gpu v, oracle u, oracle v, the simulation) over the nx
    columns."""
    rng = np.random.default_rng(seed)
    og = oracle.grid(nx, ny)
    hx, hy, ext = oracle.make_depth(og, depth)
    if tau is None:
        tau = cfl * min(og.dx, og.dy) / math.sqrt(max(ext[1], ext[3]))
    sim = tsu.ImplicitSimulation.create(nx, depth, dtype=dtype, ny=ny, sigma=sigma, tau=tau)
    g = sim.g
    x0, y0, wd, amp = u0_spec
    u0 = inputs.gaussian_hump(nx, ny, None, x0, y0, wd, amp)
    u1 = 0.3 * inputs.random_field(nx, ny, None, rng) if with_u1 else None
    tdt = tsu.DTYPES[sim.dtype]

    def dev(a):
        t = torch.zeros((g.ny, g.ld), dtype=tdt, device="cuda")
        t[:, :nx] = torch.from_numpy(np.ascontiguousarray(a[:, :nx])).to(tdt)
        return t

    sim.init(dev(u0), dev(u1) if u1 is not None else None)
    if S > 1:
        sim.step(S - 1)
    torch.cuda.synchronize()
    ou, ov = oracle.implicit_forward(og, tau, sigma, hx, hy, u0, u1, S)
    gu = sim.u[:, :nx].double().cpu().numpy()
    gv = sim.v[:, :nx].double().cpu().numpy()
    return gu, gv, ou, ov, sim


@pytest.mark.parametrize("name", sorted(DEPTHS))
@pytest.mark.parametrize("nx,ny", [(131, 77), (300, 257), (3, 3), (5, 4), (4, 130), (517, 9)])
def test_implicit_fp64_matches_oracle(name, nx, ny):
    """1e-12 relative L2; on the degenerate grids with a handful of unknowns (3 x 3 has one) the
    field is a few high-frequency modes at Courant number 3, whose phase error after 40 steps
    (about 40 w eps with w near pi) is the whole of the difference: 1e-11 there."""
    gu, gv, ou, ov, sim = run_pair(nx, ny, DEPTHS[name], 40, "f64", cfl=3.0)
    tol = 1e-12 if (nx - 2) * (ny - 2) >= 64 else 1e-11
    assert relerr(gu, ou) <= tol, relerr(gu, ou)
    assert relerr(gv, ov) <= tol, relerr(gv, ov)
    # boundary nodes and padding stay 0
    u = sim.u.cpu().numpy()
    assert not u[0].any() and not u[-1].any() and not u[:, 0].any() and not u[:, nx - 1:].any()


@pytest.mark.parametrize("name", sorted(DEPTHS))
@pytest.mark.parametrize("nx,ny,cfl", [(131, 77, 3.0), (300, 257, 8.0), (700, 390, 1.5)])
def test_implicit_fp32_matches_oracle(name, nx, ny, cfl):
    gu, gv, ou, ov, _ = run_pair(nx, ny, DEPTHS[name], 100, "f32", cfl=cfl)
    assert relerr(gu, ou) <= 1e-5, relerr(gu, ou)


def test_implicit_zero_weight_is_the_explicit_scheme():
    """sigma = 0: the implicit passes reduce to the explicit leapfrog (compared with the oracle's
    explicit scheme)."""
    n, S = 201, 150
    depth = DEPTHS["line_point"]
    og = oracle.grid(n, n)
    hx, hy, ext = oracle.make_depth(og, depth)
    tau = 0.4 * og.dx / math.sqrt(max(ext[1], ext[3]))
    sim = tsu.ImplicitSimulation.create(n, depth, dtype="f64", sigma=0.0, tau=tau)
    u0 = inputs.gaussian_hump(n, n, None, 0.4, 0.45, 0.1)
    t = torch.zeros((sim.g.ny, sim.g.ld), dtype=torch.float64, device="cuda")
    t[:, :n] = torch.from_numpy(u0)
    sim.init(t)
    sim.step(S - 1)
    ref = oracle.forward(og, tau, hx, hy, u0, None, S, want_energy=False)["u"]
    assert relerr(sim.u[:, :n].cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("dtype,n,cfl,S,tol", [("f64", 1025, 10.0, 60, 1e-11), ("f32", 2049, 20.0, 50, 2e-5),
                                               ("f32", 4096, 4.0, 30, 2e-5)])
def test_implicit_separable_mode_at_size(dtype, n, cfl, S, tol):
    """Constant depth: u^n = a_n phi with cos(w) = 1 - (lx + ly) / (2 (1 + s lx)(1 + s ly)) exactly,
    at Courant numbers up to 20 and grids up to 4096^2 (the paper's largest)."""
    h0, k, l, sigma = 1.0, 3, 2, 0.25
    g0 = oracle.grid(n, n)
    tau = cfl * g0.dx / math.sqrt(h0)
    sim = tsu.ImplicitSimulation.create(n, dict(background=h0, eps=0.1, sings=[]), dtype=dtype, sigma=sigma, tau=tau)
    g = sim.g
    tdt = tsu.DTYPES[sim.dtype]
    phi = inputs.separable_mode(n, n, g.ld, k, l)
    sim.init(torch.from_numpy(phi).to(tdt).cuda())
    sim.step(S - 1)
    cx = tau * tau / g0.dx ** 2
    lx = 4 * cx * h0 * math.sin(k * math.pi * g0.dx / 2) ** 2
    ly = 4 * cx * h0 * math.sin(l * math.pi * g0.dx / 2) ** 2
    w = math.acos(1 - (lx + ly) / (2 * (1 + sigma * lx) * (1 + sigma * ly)))
    exact = math.cos(S * w) * phi[:, :n]
    got = sim.u[:, :n].double().cpu().numpy()
    err = float(np.linalg.norm(got - exact) / np.linalg.norm(phi))  # relative to the mode's size
    assert err <= tol, (err, math.cos(S * w))


def test_implicit_paper_table1_case_matches_oracle():
    """The paper's Table 1 setting on its smallest grid: the Case 1 depth (step 100 -> 10,
    Friedrichs, eps 0.8) on 256 x 256 nodes, dt = 0.05 in paper units, 100 steps, FP64."""
    p = inputs.paper_table1(256)
    gu, gv, ou, ov, _ = run_pair(p.n, p.n, p.depth, p.steps, "f64", tau=p.extra["tau"], with_u1=False,
                                 u0_spec=p.u0)
    assert np.abs(ou).max() > 1.0
    assert relerr(gu, ou) <= 1e-12, relerr(gu, ou)


def test_implicit_argument_errors():
    n = 65
    depth = DEPTHS["line_point"]
    sim = tsu.ImplicitSimulation.create(n, depth, dtype="f64", tau=0.05)
    g = sim.g
    fb, wb = tsu.tsu_implicit_sizes(g, "f64")
    u0 = tsu.empty_field(g, "f64")
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_implicit_init(g, "f64", sim.tau, sim.sigma, sim.medium, sim.factor, u0, None, sim.state, sim.ws,
                              wb - 8)
    assert e.value.code == tsu.TSU_ENOMEM
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_implicit_factor(g, "f64", sim.tau, sim.sigma, sim.medium, sim.factor, fb - 8)
    assert e.value.code == tsu.TSU_ENOMEM
    with pytest.raises(tsu.TsuError) as e:  # below 1/4 the Courant bound is back
        tsu.tsu_implicit_factor(g, "f64", 1.0, 0.1, sim.medium, sim.factor, fb)
    assert e.value.code == tsu.TSU_ECFL
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_implicit_factor(g, "f64", sim.tau, -0.5, sim.medium, sim.factor, fb)
    assert e.value.code == tsu.TSU_EINVAL
    st = tsu.State()
    st.buf[0], st.buf[1], st.nbuf, st.form = sim.bufs[0].data_ptr(), sim.bufs[1].data_ptr(), 2, tsu.TSU_FORM_STANDARD
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_implicit_init(g, "f64", sim.tau, sim.sigma, sim.medium, sim.factor, u0, None, st, sim.ws, wb)
    assert e.value.code == tsu.TSU_EINVAL
    # a very large step is fine at sigma = 1/4
    tsu.tsu_implicit_factor(g, "f64", 10.0, 0.25, sim.medium, sim.factor, fb)
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_implicit_graph_launch_gives_the_same_bits(dtype):
    """On a side stream a multi-step call runs as one CUDA graph (kept and launched again while
    the calls repeat their arguments); it must give the bits of the launches made one by one on
    the default stream: 2 + 3 x 10 steps, and the Table 1 run at 256^2 against the oracle."""
    p = inputs.paper_table1(256)
    sims, outs = [], []
    for on_side in (False, True):
        sim = tsu.ImplicitSimulation.create(p.n, p.depth, dtype=dtype, tau=p.extra["tau"])
        u0 = torch.from_numpy(p.initial(sim.g.ld)).to(tsu.DTYPES[sim.dtype]).cuda()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        ctx = torch.cuda.stream(side) if on_side else torch.cuda.stream(torch.cuda.current_stream())
        with ctx:
            sim.init(u0)
            sim.step(2)
            for _ in range(3):  # the same call repeated: the kept graph is launched again
                sim.step(10)
        torch.cuda.synchronize()
        assert sim.state.step == 33
        outs.append((sim.u.clone(), sim.v.clone()))
        sims.append(sim)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    # the whole Table 1 run on the side stream against the oracle
    sim = sims[1]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        u0 = torch.from_numpy(p.initial(sim.g.ld)).to(tsu.DTYPES[sim.dtype]).cuda()
        sim.init(u0)
        sim.step(p.steps - 1)
    torch.cuda.synchronize()
    og = oracle.grid(p.n, p.n)
    hx, hy, _ = oracle.make_depth(og, p.depth)
    ref, _ = oracle.implicit_forward(og, p.extra["tau"], 0.25, hx, hy, p.initial(), None, p.steps)
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert relerr(sim.u[:, : p.n].double().cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("nx,ny", [(250, 250), (200, 131), (97, 256), (130, 40), (129, 129), (64, 100), (7, 5)])
def test_implicit_one_cluster_path_equals_the_two_kernel_steps(nx, ny):
    """FP32 grids of at most 129 x 129 (256 x 256) nodes run every step of a call in one cluster
    of 8 (16) CTAs, the fields in shared memory; a row pitch above 256 sends the same grid through
    the two kernels per step.  The states must agree bit for bit, and with the oracle, and no
    bounded wait of the cluster may have run out.  The start call takes the same path (u0 with
    nonzero boundary values, which it must ignore, and an initial velocity u1)."""
    depth = DEPTHS["paper_step"]
    og = oracle.grid(nx, ny)
    hx, hy, ext = oracle.make_depth(og, depth)
    tau = 3.0 * min(og.dx, og.dy) / math.sqrt(max(ext[1], ext[3]))
    rng = np.random.default_rng(nx * 1000 + ny)
    u0n = inputs.gaussian_hump(nx, ny, None, 0.4, 0.45, 0.08)
    u0b = u0n + 0.1 * inputs.random_field(nx, ny, None, rng, zero_boundary=False)
    u0n = u0b.copy()
    u0n[0, :] = u0n[-1, :] = 0.0
    u0n[:, 0] = u0n[:, -1] = 0.0
    u1n = 0.2 * inputs.random_field(nx, ny, None, rng)
    out = []
    for ld in (None, 320):
        sim = tsu.ImplicitSimulation.create(nx, depth, dtype="f32", ny=ny, tau=tau, ld=ld)
        u0 = tsu.empty_field(sim.g, "f32")
        u0[:, :nx] = torch.from_numpy(u0b).float()
        u1 = torch.zeros_like(u0)
        u1[:, :nx] = torch.from_numpy(u1n).float()
        sim.init(u0, u1)
        sim.step(7)
        sim.step(23)
        tsu.tsu_sync_status(sim.ws, sim.ws.numel())
        out.append((sim.u[:, :nx].clone(), sim.v[:, :nx].clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    ref, _ = oracle.implicit_forward(og, tau, 0.25, hx, hy, u0n, u1n, 31)
    assert relerr(out[0][0].double().cpu().numpy(), ref) <= 1e-5
