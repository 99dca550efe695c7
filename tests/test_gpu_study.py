"""GPU tests of the eps-family tools: d h_eps / d eps at the faces, its contraction with adjoint
face gradients (dJ/deps), the field-difference norms, and the study drivers built on them.

d h / d eps and the norms are compared with the oracle (numpy sums of oracle fields); dJ/deps with
central differences of J(eps) computed by the oracle's forward map; the drivers with the paper's
claims (Sec. 3.2: the regularised family converges as eps -> 0 and does not depend on the choice
of mollifier in the limit).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2005_11931_gb300 import inputs, study, tsu
from tests.gpu_helpers import relerr
from tests.test_oracle_pins import EPS_DEPTHS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", sorted(EPS_DEPTHS))
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-6)])
def test_depth_eps_derivative_matches_oracle(name, dtype, tol):
    depth = EPS_DEPTHS[name]
    nx, ny = 301, 197
    g = tsu.grid(nx, ny)
    dhx = tsu.empty_field(g, dtype)
    dhy = tsu.empty_field(g, dtype)
    tsu.tsu_depth_eps_derivative(g, depth, dtype, dhx, dhy)
    og = oracle.grid(nx, ny)
    ox, oy = oracle.depth_deps(og, depth)
    torch.cuda.synchronize()
    assert relerr(dhx[:, :nx].double().cpu().numpy(), ox) <= tol
    assert relerr(dhy[:, :nx].double().cpu().numpy(), oy) <= tol
    # entries outside the faces are 0
    assert float(dhx[:, nx - 1:].abs().max()) == 0.0
    assert float(dhy[ny - 1:, :].abs().max()) == 0.0


def test_eps_gradient_is_the_contraction_with_the_oracle_derivative():
    depth = EPS_DEPTHS["point_gauss"]
    nx, ny = 333, 250
    g = tsu.grid(nx, ny)
    rng = np.random.default_rng(5)
    gx = np.zeros((ny, g.ld))
    gy = np.zeros((ny, g.ld))
    gx[:, : nx - 1] = rng.standard_normal((ny, nx - 1))
    gy[: ny - 1, :nx] = rng.standard_normal((ny - 1, nx))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(tsu.tsu_reduce_workspace(), dtype=torch.uint8, device="cuda")
    tsu.tsu_depth_eps_gradient(g, depth, torch.from_numpy(gx).cuda(), torch.from_numpy(gy).cuda(), out, ws)
    ox, oy = oracle.depth_deps(oracle.grid(nx, ny), depth)
    ref = float(np.sum(gx[:, :nx] * ox) + np.sum(gy[:, :nx] * oy))
    assert abs(float(out) - ref) <= 1e-11 * (np.sum(np.abs(gx[:, :nx] * ox)) + np.sum(np.abs(gy[:, :nx] * oy)))
    # deterministic: the same bits again
    out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    tsu.tsu_depth_eps_gradient(g, depth, torch.from_numpy(gx).cuda(), torch.from_numpy(gy).cuda(), out2, ws)
    assert float(out2) == float(out)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_diff_norms_match_numpy(dtype):
    nx, ny = 1001, 517
    g = tsu.grid(nx, ny)
    rng = np.random.default_rng(9)
    a = tsu.empty_field(g, dtype)
    b = tsu.empty_field(g, dtype)
    a[:, :nx] = torch.from_numpy(rng.standard_normal((ny, nx))).to(a.dtype)
    b[:, :nx] = torch.from_numpy(rng.standard_normal((ny, nx))).to(b.dtype)
    b[:, nx:] = 7.0  # padding is outside the grid: not counted
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    ws = torch.empty(tsu.tsu_reduce_workspace(), dtype=torch.uint8, device="cuda")
    tsu.tsu_diff_norms(g, dtype, a, b, out, ws)
    an = a[:, :nx].double().cpu().numpy()
    bn = b[:, :nx].double().cpu().numpy()
    ref = np.array([np.sum((an - bn) ** 2), np.sum(bn ** 2)])
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_misfit_eps_gradient_matches_central_differences():
    """dJ/deps through the adjoint's face gradients and d h / d eps, for a receiver misfit on a
    line singularity, against central differences of J(eps) with the oracle's forward map."""
    n, S = 97, 160
    base = dict(background=1.0, eps=0.04, mollifier=0, sings=[(0, 1, 0.5, 0.5, 0.5)])
    rng = np.random.default_rng(inputs.SEED)
    rec_ij = inputs.receivers_on_row(n, 0.7, 12, rng)
    u0 = inputs.gaussian_hump(n, n, None, 0.35, 0.6, 0.06)
    res = study.misfit_eps_gradient(n, base, u0, S, rec_ij, eps_obs=0.05, dtype="f64", ckpt_every=16)
    og = oracle.grid(n, n)
    ridx = inputs.flat_index(rec_ij, n)

    def J(eps):
        hx, hy, _ = oracle.make_depth(og, dict(base, eps=eps))
        tr = oracle.forward(og, res["tau"], hx, hy, u0[:, :n], None, S, want_energy=False, rec_idx=ridx)["traces"]
        return 0.5 * float(np.sum((tr - res["observed"]) ** 2))

    assert abs(J(base["eps"]) / res["J"] - 1) < 1e-10
    st = 1e-5
    fd = (J(base["eps"] + st) - J(base["eps"] - st)) / (2 * st)
    assert abs(res["dJ_deps"] - fd) <= 1e-6 * abs(fd), (res["dJ_deps"], fd)


def test_eps_family_converges_as_eps_decreases():
    """Sec. 3.2: the regularised solutions form a Cauchy family as eps -> 0; the relative
    difference between neighbours of a halving sequence decreases."""
    r = study.eps_convergence("line_x", [0.064, 0.032, 0.016, 0.008], n=1025, T=0.15)
    d = r["relative_differences"]
    assert len(d) == 3
    assert all(d[k + 1] < d[k] for k in range(len(d) - 1)), d
    assert d[0] > 0


def test_mollifier_choice_fades_as_eps_decreases():
    """Sec. 3.2: the limit does not depend on the mollifier; the Gaussian and Friedrichs families at
    the same eps get closer as eps decreases."""
    r = study.mollifier_gap([0.064, 0.032, 0.016], n=1025, T=0.15)
    g = r["relative_gaps"]
    assert all(g[k + 1] < g[k] for k in range(len(g) - 1)), g


def test_reflected_pulse_from_a_line_singularity():
    """Sec. 3.2: a wave meeting the line singularity is partly reflected.  The receiver between
    the source and the line sees the free wave first; the difference to the run without the line
    arrives after the time to the line and back (0.2 + 0.1 at speed 1, less the line's width), is
    a fraction of the incident pulse, and its size settles as eps decreases."""
    r = [study.reflected_pulse(e, n=769, T=0.45) for e in (0.02, 0.01)]
    for q in r:
        assert q["incident_peak"] > 0 and abs(q["incident_arrival"] - 0.1) < 0.03
        assert 0.2 < q["reflected_arrival"] < 0.32
        assert 1e-2 * q["incident_peak"] < abs(q["reflected_peak"]) < q["incident_peak"]
    assert np.sign(r[0]["reflected_peak"]) == np.sign(r[1]["reflected_peak"])
    assert abs(r[1]["reflected_peak"] / r[0]["reflected_peak"] - 1) < 0.5


def test_argument_errors_of_the_study_entry_points():
    g = tsu.grid(65, 65)
    depth = EPS_DEPTHS["line_gauss"]
    f = tsu.empty_field(g, "f64")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    ws = torch.empty(tsu.tsu_reduce_workspace(), dtype=torch.uint8, device="cuda")
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_diff_norms(g, "f64", f, f, out, small)
    assert e.value.code == tsu.TSU_ENOMEM
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_depth_eps_gradient(g, depth, f, f, out, small)
    assert e.value.code == tsu.TSU_ENOMEM
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_depth_eps_derivative(g, dict(depth, eps=-1.0), "f64", f, f)
    assert e.value.code == tsu.TSU_EINVAL
    # a misaligned field is refused too: checked without a device (tests/host_checks.py)
