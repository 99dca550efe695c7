"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Every check here compares the oracle with something other than
itself: a closed-form discrete solution, d'Alembert's formula, an eigen-
decomposition, calculus (convergence order), quadrature by scipy, an invariant,
or finite differences of the oracle's own forward map (for the adjoint).
A plausible slip in the oracle -- a dropped term, a face index off by one, a
wrong sign, a transposed operand, a missing 1/2 -- fails at least one test.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2005_11931_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# Mollifier (Sec. 2.1 regularisation; Sec. 3.1 Friedrichs bump)
# ---------------------------------------------------------------------------
def test_friedrichs_constant_matches_paper_and_quadrature():
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["friedrichs_c"]
    c1, c2 = oracle.friedrichs_constants()
    assert abs(c1 - gold["value"]) < 0.5 * 10 ** -gold["digits"]
    bump = lambda x: math.exp(1.0 / (x * x - 1.0)) if abs(x) < 1 else 0.0
    mass1, _ = integrate.quad(bump, -1, 1, epsabs=1e-15, epsrel=1e-14, limit=200)
    assert abs(c1 * mass1 - 1.0) < 1e-12
    mass2, _ = integrate.quad(lambda r: 2 * math.pi * r * bump(r), 0, 1, epsabs=1e-15, epsrel=1e-14, limit=200)
    assert abs(c2 * mass2 - 1.0) < 1e-12


@pytest.mark.parametrize("moll,eps_cells,tol", [(inputs.GAUSS, 3.0, 1e-9), (inputs.GAUSS, 6.5, 1e-9),
                                               (inputs.FRIEDRICHS, 40.0, 1e-8)])
def test_line_mollifier_unit_mass_and_width(moll, eps_cells, tol):
    """Unit mass, centre and width of the 1D mollifier.  The Riemann sum of the Gaussian is exact
    to ~exp(-pi^2 eps^2/dx^2); the compactly supported bump converges more slowly, so it is
    checked at a width of 40 cells."""
    n = 801
    g = oracle.grid(n, 9)
    eps = eps_cells * g.dx
    c = 0.5 + 0.3 * g.dx  # off-node centre
    hx, hy, ext = oracle.make_depth(g, dict(background=0.0, eps=eps, mollifier=moll,
                                            sings=[(inputs.LINE_X, 1, 1.0, c, 0.5)]))
    # hy is sampled at x_i (nodes): a Riemann sum of phi_eps(x - c)
    row = hy[3, :n]
    x = np.arange(n) * g.dx
    mass = row.sum() * g.dx
    assert abs(mass - 1.0) < tol
    # first moment = c (symmetric bump), second central moment fixes the width convention
    m1 = (row * x).sum() * g.dx
    assert abs(m1 - c) < tol
    var = (row * (x - c) ** 2).sum() * g.dx
    if moll == inputs.GAUSS:
        expect = eps ** 2 / 2.0  # exp(-s^2/eps^2)/(eps sqrt(pi)) has variance eps^2/2
    else:
        bump = lambda t: math.exp(1.0 / (t * t - 1.0)) if abs(t) < 1 else 0.0
        c1 = 1.0 / integrate.quad(bump, -1, 1, epsabs=1e-15, epsrel=1e-14)[0]
        expect = eps ** 2 * c1 * integrate.quad(lambda t: t * t * bump(t), -1, 1, epsabs=1e-15)[0]
    assert abs(var / expect - 1.0) < 1e-6 if moll == inputs.GAUSS else abs(var / expect - 1.0) < 1e-5
    # line in x: h does not depend on y; the y-direction faces are unused rows
    assert np.all(hy[:-1, :n] == hy[3, :n])


@pytest.mark.parametrize("moll,eps_cells", [(inputs.GAUSS, 5.0), (inputs.FRIEDRICHS, 40.0)])
def test_point_mollifier_unit_mass(moll, eps_cells):
    """Unit mass of the 2D point mollifier (eps^-2 scaling in two dimensions)."""
    n = 161
    g = oracle.grid(n, n)
    eps = eps_cells * g.dx
    hx, hy, ext = oracle.make_depth(g, dict(background=0.0, eps=eps, mollifier=moll,
                                            sings=[(inputs.POINT, 1, 1.0, 0.43, 0.57)]))
    assert abs(hx.sum() * g.dx * g.dy - 1.0) < 1e-9
    assert abs(hy.sum() * g.dx * g.dy - 1.0) < 1e-9
    # peak of a unit-mass 2D Gaussian of width eps is 1/(pi eps^2); faces sit near the centre
    if moll == inputs.GAUSS:
        assert ext[1] <= 1.0 / (math.pi * eps * eps) * (1 + 1e-14)
        assert ext[1] > 0.9 / (math.pi * eps * eps)


def test_delta_squared_power():
    """Case 3 of Sec. 3.1: delta^2 regularised as phi_eps^2.  For the Gaussian,
    int phi_eps^2 = 1/(eps sqrt(2 pi))."""
    n = 801
    g = oracle.grid(n, 5)
    eps = 8 * g.dx
    _, hy, _ = oracle.make_depth(g, dict(background=0.0, eps=eps, sings=[(inputs.LINE_X, 2, 1.0, 0.5, 0.5)]))
    assert abs(hy[2, :n].sum() * g.dx * eps * math.sqrt(2 * math.pi) - 1.0) < 1e-9


@pytest.mark.parametrize("moll", [inputs.GAUSS, inputs.FRIEDRICHS])
def test_step_is_integral_of_line(moll):
    """Case 1 of Sec. 3.1 (the step h0 mollified): the mollified Heaviside's x-derivative
    is minus the mollified delta of the same width; the step is amp on the left, 0 on the right,
    amp/2 at the jump."""
    n = 1001
    g = oracle.grid(n, 5)
    eps = 0.02
    cstep = 0.6
    d_step = dict(background=0.0, eps=eps, mollifier=moll, sings=[(inputs.STEP_X, 1, 90.0, cstep, 0.5)])
    d_line = dict(background=0.0, eps=eps, mollifier=moll, sings=[(inputs.LINE_X, 1, 90.0, cstep, 0.5)])
    _, hy_s, _ = oracle.make_depth(g, d_step)
    hx_l, _, _ = oracle.make_depth(g, d_line)
    s = hy_s[2, :n]           # step at nodes x_i
    dline = hx_l[2, : n - 1]  # delta at faces x_i + dx/2
    deriv = (s[1:] - s[:-1]) / g.dx
    assert np.max(np.abs(deriv + dline)) < 2e-3 * np.max(dline)
    assert abs(s[0] - 90.0) < 1e-12 and abs(s[-1]) < 1e-12
    assert abs(s[600] - 45.0) < 1e-9  # node 600 sits at x = 0.6


def test_config1_peak_depth():
    """201^2 line case: hy faces sit on x = 0.5 exactly, so max h = 1 + 1/(eps sqrt(pi))."""
    p = inputs.line_fp64_201()
    g = oracle.grid(p.n, p.n)
    _, _, ext = oracle.make_depth(g, p.depth)
    assert abs(ext[3] - (1 + 1 / (0.02 * math.sqrt(math.pi)))) < 1e-12
    assert ext[0] == 1.0 and ext[2] == 1.0


# ---------------------------------------------------------------------------
# Time stepping: exact discrete solutions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,k,l,S,h0,v", [
    (33, 33, 1, 1, 400, 1.0, 0.0),
    (41, 29, 3, 2, 700, 2.5, 0.0),
    (41, 29, 2, 5, 300, 0.7, 1.3),
    (17, 65, 7, 1, 900, 1.0, -0.4),
])
def test_separable_mode_exact(nx, ny, k, l, S, h0, v):
    """Constant depth h0: sin(k pi x) sin(l pi y) is an eigenvector of the discrete operator with
    lambda = 4h0/dx^2 sin^2(k pi dx/2) + 4h0/dy^2 sin^2(l pi dy/2).  With u0 = phi, u1 = v phi the
    scheme (Taylor start included) gives u^n = [cos(n theta) + tau v sin(n theta)/sin(theta)] phi,
    cos(theta) = 1 - tau^2 lambda / 2."""
    g = oracle.grid(nx, ny)
    hx, hy, ext = oracle.make_depth(g, dict(background=h0, eps=0.1, sings=[]))
    tau = 0.4 * min(g.dx, g.dy) / math.sqrt(h0)
    phi = inputs.separable_mode(nx, ny, None, k, l)
    lam = 4 * h0 / g.dx ** 2 * math.sin(k * math.pi * g.dx / 2) ** 2 + 4 * h0 / g.dy ** 2 * math.sin(
        l * math.pi * g.dy / 2) ** 2
    theta = math.acos(1 - tau * tau * lam / 2)
    out = oracle.forward(g, tau, hx, hy, phi, v * phi, S, rec_idx=None)
    for n, u in ((S - 1, out["u_prev"]), (S, out["u"])):
        coef = math.cos(n * theta) + tau * v * math.sin(n * theta) / math.sin(theta)
        exact = coef * phi
        assert np.max(np.abs(u - exact)) < 1e-11 * max(1.0, abs(coef)), (n, np.max(np.abs(u - exact)))
    # discrete energy of the mode: with ||phi||^2 dxdy = 1/4,
    # E^{n+1/2} = 1/8 [ ((a_{n+1}-a_n)/tau)^2 + lambda a_{n+1} a_n ]
    a = lambda n: math.cos(n * theta) + tau * v * math.sin(n * theta) / math.sin(theta)
    for n in (0, S // 3, S - 1):
        e = out["energy"][n]
        ex = 0.125 * (((a(n + 1) - a(n)) / tau) ** 2 + lam * a(n + 1) * a(n))
        assert abs(e - ex) < 1e-11 * abs(ex), (n, e, ex)


def test_dispersion_relation_converges():
    """theta/tau -> pi sqrt(h0 (k^2 + l^2)) as dx -> 0 (continuous dispersion), measured on the
    oracle's trajectory by the phase at a fixed time."""
    h0, k, l, T = 1.3, 2, 1, 0.15
    errs = []
    for n in (17, 33, 65):
        g = oracle.grid(n, n)
        hx, hy, _ = oracle.make_depth(g, dict(background=h0, eps=0.1, sings=[]))
        S = 8 * (n - 1)
        tau = T / S
        phi = inputs.separable_mode(n, n, None, k, l)
        u = oracle.forward(g, tau, hx, hy, phi, None, S, want_energy=False)["u"]
        i, j = (n - 1) // 4, (n - 1) // 2 - 1
        ratio = u[j, i] / phi[j, i]
        exact = math.cos(math.pi * math.sqrt(h0 * (k * k + l * l)) * T)
        errs.append(abs(ratio - exact))
    # second order in space and time
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def odd_periodic(f):
    """Odd 2(N-1)-periodic extension of node data f[0..N-1] with f[0] = f[N-1] = 0."""
    return np.concatenate([f, -f[-2:0:-1]])


@pytest.mark.parametrize("S", [1, 2, 37, 300])
def test_dalembert_courant_one_bit_exact(S):
    """Sec. 3.3 box with hy = 0, hx = 1 and tau = dx: the scheme is exactly d'Alembert's formula
    u(x,t) = (f(x-t) + f(x+t))/2 with odd reflection at the Dirichlet ends (u1 = 0)."""
    nx, ny = 129, 6
    g = oracle.grid(nx, ny)
    hx = np.zeros((ny, nx))
    hx[:, : nx - 1] = 1.0
    hy = np.zeros((ny, nx))
    tau = g.dx  # dx = 2^-7: tau^2/dx^2 = 1 exactly
    rng = np.random.default_rng(3)
    u0 = np.zeros((ny, nx))
    u0[1:-1, 1:-1] = 2.0 * rng.integers(-50, 50, size=(ny - 2, nx - 2))
    out = oracle.forward(g, tau, hx, hy, u0, None, S, want_energy=False)
    for j in range(1, ny - 1):
        F = odd_periodic(u0[j])
        P = len(F)
        idx = np.arange(nx)
        exact = 0.5 * (F[(idx - S) % P] + F[(idx + S) % P])
        assert np.array_equal(out["u"][j], exact)


def test_spectral_solution_variable_depth():
    """Tiny grid, variable depth: with B = V diag(mu) V^T (B = tau^2 L_h assembled column by column
    from the oracle's operator), the scheme's solution is u^n = V [cos(n theta) c0 +
    tau sin(n theta)/sin(theta) c1], cos(theta) = 1 + mu/2, c = V^T u."""
    nx, ny = 9, 7
    g = oracle.grid(nx, ny)
    depth = dict(background=0.3, eps=0.15, sings=[(inputs.POINT, 1, 0.2, 0.3, 0.6),
                                                  (inputs.LINE_X, 1, 0.5, 0.55, 0.5),
                                                  (inputs.LINE_Y, 1, 0.3, 0.5, 0.35)])
    hx, hy, ext = oracle.make_depth(g, depth)
    tau = 0.4 / math.sqrt(ext[1] / g.dx ** 2 + ext[3] / g.dy ** 2)
    interior = [(j, i) for j in range(1, ny - 1) for i in range(1, nx - 1)]
    m = len(interior)
    Bm = np.zeros((m, m))
    for c, (j, i) in enumerate(interior):
        e = np.zeros((ny, nx))
        e[j, i] = 1.0
        Be = oracle.apply_B(g, tau, hx, hy, e)
        Bm[:, c] = [Be[jj, ii] for (jj, ii) in interior]
    assert np.array_equal(Bm, Bm.T)  # symmetric (self-adjoint face form)
    mu, V = np.linalg.eigh(Bm)
    assert mu.max() < 0 and mu.min() > -4.0  # negative definite, inside the leapfrog bound
    theta = np.arccos(1 + mu / 2)
    rng = np.random.default_rng(11)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    vec = lambda f: np.array([f[j, i] for (j, i) in interior])
    c0, c1 = V.T @ vec(u0), V.T @ vec(u1)
    for S in (1, 2, 5, 60):
        out = oracle.forward(g, tau, hx, hy, u0, u1, S, want_energy=False)
        exact = V @ (np.cos(S * theta) * c0 + tau * np.sin(S * theta) / np.sin(theta) * c1)
        assert np.max(np.abs(vec(out["u"]) - exact)) < 1e-12 * np.max(np.abs(exact)) * 10, S


# ---------------------------------------------------------------------------
# Operator: consistency with d_x(h d_x u) + d_y(h d_y u) (eq. (2.1))
# ---------------------------------------------------------------------------
def test_operator_second_order_consistency():
    """(B u)/tau^2 -> d_x(h d_x u) + d_y(h d_y u) at second order for smooth h and u; a face
    sampled at the node instead of the face, or a wrong 1/dx^2, breaks the order or the limit."""
    eps, a, b = 0.12, 0.7, 0.4
    gph = lambda s: math.exp(-(s / eps) ** 2) / (eps * math.sqrt(math.pi))
    h = lambda x, y: 1.0 + a * gph(x - 0.45) + b * gph(y - 0.6)
    hxd = lambda x, y: a * gph(x - 0.45) * (-2 * (x - 0.45) / eps ** 2)
    hyd = lambda x, y: b * gph(y - 0.6) * (-2 * (y - 0.6) / eps ** 2)
    u = lambda x, y: math.sin(math.pi * x) * math.sin(2 * math.pi * y) * math.exp(x * y)
    ux = lambda x, y: (math.pi * math.cos(math.pi * x) + y * math.sin(math.pi * x)) * math.sin(
        2 * math.pi * y) * math.exp(x * y)
    uy = lambda x, y: (2 * math.pi * math.cos(2 * math.pi * y) + x * math.sin(2 * math.pi * y)) * math.sin(
        math.pi * x) * math.exp(x * y)

    def uxx(x, y):
        s, c, e = math.sin(math.pi * x), math.cos(math.pi * x), math.exp(x * y)
        return (-math.pi ** 2 * s + 2 * y * math.pi * c + y * y * s) * math.sin(2 * math.pi * y) * e

    def uyy(x, y):
        s, c, e = math.sin(2 * math.pi * y), math.cos(2 * math.pi * y), math.exp(x * y)
        return (-4 * math.pi ** 2 * s + 4 * x * math.pi * c + x * x * s) * math.sin(math.pi * x) * e

    errs = []
    for n in (41, 81, 161):
        g = oracle.grid(n, n)
        hx, hy, _ = oracle.make_depth(g, dict(background=1.0, eps=eps, sings=[(inputs.LINE_X, 1, a, 0.45, 0.5),
                                                                              (inputs.LINE_Y, 1, b, 0.5, 0.6)]))
        tau = 0.1 * g.dx
        uu = np.array([[u(i * g.dx, j * g.dy) for i in range(n)] for j in range(n)])
        uu[0, :] = uu[-1, :] = 0
        uu[:, 0] = uu[:, -1] = 0
        Lu = oracle.apply_B(g, tau, hx, hy, uu) / tau ** 2
        exact = np.array([[hxd(i * g.dx, j * g.dy) * ux(i * g.dx, j * g.dy) + h(i * g.dx, j * g.dy) * uxx(
            i * g.dx, j * g.dy) + hyd(i * g.dx, j * g.dy) * uy(i * g.dx, j * g.dy) + h(i * g.dx, j * g.dy) * uyy(
            i * g.dx, j * g.dy) for i in range(n)] for j in range(n)])
        errs.append(np.max(np.abs(Lu - exact)[1:-1, 1:-1]))
    assert errs[0] / errs[1] > 3.6 and errs[1] / errs[2] > 3.6, errs


# ---------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------
def test_energy_conserved_variable_depth():
    """Leapfrog analogue of (CL-01), Theorem 2.1: E^{n+1/2} is constant up to round-off for any
    positive face depth under the CFL bound, with nonzero initial velocity."""
    n = 97
    g = oracle.grid(n, n - 16)
    depth = dict(background=0.8, eps=0.03, sings=[(inputs.POINT, 1, 0.004, 0.4, 0.45),
                                                  (inputs.LINE_X, 1, 0.6, 0.62, 0.5)])
    hx, hy, ext = oracle.make_depth(g, depth)
    tau = 0.9 / math.sqrt(ext[1] / g.dx ** 2 + ext[3] / g.dy ** 2)
    u0 = inputs.gaussian_hump(g.nx, g.ny, None, 0.3, 0.5, 0.08)
    u1 = 0.5 * inputs.gaussian_hump(g.nx, g.ny, None, 0.5, 0.4, 0.1)
    out = oracle.forward(g, tau, hx, hy, u0, u1, 1000)
    E = out["energy"]
    assert E.min() > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12


def test_energy_not_conserved_by_a_wrong_face_index():
    """Sanity of the invariant test itself: shifting hx by one face (a plausible indexing slip)
    in the energy breaks conservation by far more than round-off."""
    n = 65
    g = oracle.grid(n, n)
    depth = dict(background=0.8, eps=0.05, sings=[(inputs.LINE_X, 1, 0.6, 0.52, 0.5)])
    hx, hy, ext = oracle.make_depth(g, depth)
    tau = 0.5 / math.sqrt(ext[1] / g.dx ** 2 + ext[3] / g.dy ** 2)
    u0 = inputs.gaussian_hump(n, n, None, 0.35, 0.5, 0.08)
    out = oracle.forward(g, tau, hx, hy, u0, None, 400)
    hx_bad = np.roll(hx, 1, axis=1)
    up, uc = oracle.init(g, tau, hx, hy, u0)
    e0 = oracle.energy(g, tau, hx_bad, hy, up, uc)
    e1 = oracle.energy(g, tau, hx_bad, hy, out["u_prev"], out["u"])
    assert abs(e1 - e0) / e0 > 1e-4
    assert np.max(np.abs(out["energy"] - out["energy"][0])) / out["energy"][0] < 1e-12


def test_mirror_symmetry_line_case():
    """The 201^2 line case has y -> 1-y symmetry (h independent of y, hump centred at y = 0.5):
    the solution is mirror symmetric bit for bit."""
    p = inputs.line_fp64_201()
    n = 101
    g = oracle.grid(n, n)
    hx, hy, ext = oracle.make_depth(g, p.depth)
    tau = 0.4 * g.dx / math.sqrt(max(ext[1], ext[3]))
    u0 = inputs.gaussian_hump(n, n, None, 0.25, 0.5, 0.05)
    out = oracle.forward(g, tau, hx, hy, u0, None, 300, want_energy=False)
    assert np.array_equal(out["u"], out["u"][::-1, :])
    assert np.abs(out["u"]).max() > 0.05


# ---------------------------------------------------------------------------
# Discrete adjoint (not in the paper): finite differences of the forward map
# ---------------------------------------------------------------------------
def test_adjoint_matches_central_differences():
    nx, ny, S = 12, 10, 40
    g = oracle.grid(nx, ny)
    depth = dict(background=0.9, eps=0.12, sings=[(inputs.POINT, 1, 0.05, 0.4, 0.5),
                                                  (inputs.LINE_X, 1, 0.3, 0.6, 0.5)])
    hx, hy, ext = oracle.make_depth(g, depth)
    tau = 0.45 / math.sqrt(ext[1] / g.dx ** 2 + ext[3] / g.dy ** 2)
    rng = np.random.default_rng(5)
    u0 = inputs.random_field(nx, ny, None, rng)
    u1 = inputs.random_field(nx, ny, None, rng)
    # receivers: distinct interior nodes, one duplicate, one on the boundary
    rec = np.array([3 * nx + 4, 5 * nx + 7, 7 * nx + 2, 5 * nx + 7, 0 * nx + 5], dtype=np.int64)
    d = rng.standard_normal((S, len(rec)))

    def J(hx_, hy_, u0_, u1_):
        tr = oracle.forward(g, tau, hx_, hy_, u0_, u1_, S, want_energy=False, rec_idx=rec)["traces"]
        return 0.5 * np.sum((tr - d) ** 2), tr

    J0, tr = J(hx, hy, u0, u1)
    grads = oracle.adjoint(g, tau, hx, hy, u0, u1, S, rec, tr - d)
    facemask_x = np.zeros((ny, nx), bool)
    facemask_x[:, : nx - 1] = True
    facemask_y = np.zeros((ny, nx), bool)
    facemask_y[: ny - 1, :] = True
    for name, base, mask in (("g_hx", hx, facemask_x), ("g_hy", hy, facemask_y),
                             ("g_u0", u0, np.ones((ny, nx), bool)), ("g_u1", u1, np.ones((ny, nx), bool))):
        for trial in range(3):
            dirn = rng.standard_normal((ny, nx)) * mask
            if name in ("g_hx", "g_hy"):
                dirn *= 0.1
            step = 1e-5
            args = dict(g_hx=(hx, hy, u0, u1), g_hy=(hx, hy, u0, u1), g_u0=(hx, hy, u0, u1),
                        g_u1=(hx, hy, u0, u1))[name]
            pos = list(args)
            neg = list(args)
            k = ["g_hx", "g_hy", "g_u0", "g_u1"].index(name)
            pos[k] = base + step * dirn
            neg[k] = base - step * dirn
            fd = (J(*pos)[0] - J(*neg)[0]) / (2 * step)
            ad = float(np.sum(grads[name] * dirn))
            assert abs(fd - ad) <= 1e-7 * max(1.0, abs(fd)), (name, fd, ad)
    # gradients vanish where the variable has no effect
    assert np.all(grads["g_u0"][0, :] == 0) and np.all(grads["g_u1"][:, 0] == 0)
    assert np.all(grads["g_hx"][0, :] == 0) and np.all(grads["g_hx"][:, nx - 1] == 0)


# ---------------------------------------------------------------------------
# The paper's claim: the regularised family is Cauchy as eps -> 0 (Sec. 3.2)
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_eps_family_is_cauchy():
    """Sec. 3.2 (limiting behaviour, irregular case): ||u_eps1 - u_eps2|| -> 0 as eps1, eps2 -> 0
    for a line delta in the depth.  Checked as a monotone decrease of d(eps) = ||u_eps - u_eps/2||
    at a fixed time on a fixed grid (parity unpinned beyond monotone decrease)."""
    n = 201
    g = oracle.grid(n, n)
    eps_list = [0.08, 0.04, 0.02]
    depths = [dict(background=1.0, eps=e, sings=[(inputs.LINE_X, 1, 0.2, 0.5, 0.5)]) for e in eps_list + [0.01]]
    exts = [oracle.make_depth(g, d) for d in depths]
    hmax = max(max(e[2][1], e[2][3]) for e in exts)
    tau = 0.4 * g.dx / math.sqrt(hmax)
    T = 0.35
    S = int(round(T / tau))
    u0 = inputs.gaussian_hump(n, n, None, 0.25, 0.5, 0.05)
    sols = [oracle.forward(g, tau, hx, hy, u0, None, S, want_energy=False)["u"] for hx, hy, _ in exts]
    d = [np.linalg.norm(sols[k] - sols[k + 1]) * g.dx for k in range(3)]
    assert d[0] > d[1] > d[2], d


EPS_DEPTHS = {
    "line_gauss": dict(background=1.0, eps=0.03, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5)]),
    "line_y_friedrichs": dict(background=1.0, eps=0.05, mollifier=1, sings=[(1, 1, 0.7, 0.5, 0.43)]),
    "point_gauss": dict(background=0.5, eps=0.04, mollifier=0, sings=[(2, 1, 0.01, 0.47, 0.52)]),
    "point_friedrichs": dict(background=0.5, eps=0.06, mollifier=1, sings=[(2, 1, 0.01, 0.5, 0.5)]),
    "delta2": dict(background=1.0, eps=0.05, mollifier=0, sings=[(1, 2, 0.002, 0.5, 0.6)]),
    "step_gauss": dict(background=10.0, eps=0.02, mollifier=0, sings=[(3, 1, 90.0, 0.75, 0.5)]),
    "step_friedrichs_y": dict(background=2.0, eps=0.04, mollifier=1, sings=[(4, 1, 3.0, 0.5, 0.33)]),
}


@pytest.mark.parametrize("name", sorted(EPS_DEPTHS))
def test_depth_eps_derivative_matches_central_differences(name):
    """d h_eps / d eps (the analytic derivative of Sec. 2.1's regularisation in its width) against
    central differences of the face depth in eps, for every singularity kind, both mollifiers and
    the delta^2 power."""
    depth = EPS_DEPTHS[name]
    g = oracle.grid(97, 89)
    dhx, dhy = oracle.depth_deps(g, depth)
    eps, st = depth["eps"], 1e-5 * depth["eps"]
    hp = oracle.make_depth(g, dict(depth, eps=eps + st))
    hm = oracle.make_depth(g, dict(depth, eps=eps - st))
    fdx, fdy = (hp[0] - hm[0]) / (2 * st), (hp[1] - hm[1]) / (2 * st)
    assert np.abs(dhx).max() + np.abs(dhy).max() > 0
    assert relerr(dhx, fdx) <= 1e-7, relerr(dhx, fdx)
    assert relerr(dhy, fdy) <= 1e-7, relerr(dhy, fdy)


@pytest.mark.parametrize("moll", [0, 1])
def test_depth_eps_derivative_keeps_the_mass(moll):
    """A unit-mass mollifier keeps unit mass at every width, so d/deps of its integral is 0: the
    face sums of d h / d eps vanish for a line (1D sum across it) and a point (2D sum).  The
    bump's derivative is steep near the edge of its support, so it gets a wider eps (the sums
    converge spectrally: 1.2e-3, 4e-6, 8e-9, 2e-11 at eps = 0.02, 0.05, 0.1, 0.15 on this grid)."""
    n = 801
    g = oracle.grid(n, n)
    eps = 0.02 if moll == 0 else 0.15
    line = dict(background=1.0, eps=eps, mollifier=moll, sings=[(0, 1, 1.0, 0.5, 0.5)])
    dhx, _ = oracle.depth_deps(g, line)
    row = dhx[n // 2, : n - 1]
    assert abs(row.sum() * g.dx) <= 1e-9 * np.abs(row).sum() * g.dx
    point = dict(background=1.0, eps=1.5 * eps, mollifier=moll, sings=[(2, 1, 1.0, 0.5, 0.5)])
    _, dhy = oracle.depth_deps(g, point)
    tot = dhy[: n - 1, :n]
    assert abs(tot.sum()) <= 1e-8 * np.abs(tot).sum()


@pytest.mark.parametrize("increment", [False, True])
def test_fp32_emulation_is_exact_at_courant_one(increment):
    """The oracle's FP32 mode is pinned like its FP64 one: at Courant 1 in x (hy = 0, tau = dx,
    even integer data) every operation is exact in FP32 as well, so both forms reproduce
    d'Alembert's solution bit for bit."""
    nx, ny, S = 129, 6, 77
    g = oracle.grid(nx, ny)
    hx = np.zeros((ny, nx))
    hx[:, : nx - 1] = 1.0
    hy = np.zeros((ny, nx))
    rng = np.random.default_rng(4)
    u0 = np.zeros((ny, nx))
    u0[1:-1, 1:-1] = 2.0 * rng.integers(-50, 50, size=(ny - 2, nx - 2))
    out = oracle.forward_f32(g, g.dx, hx, hy, u0, None, S, increment)
    for j in range(1, ny - 1):
        F = odd_periodic(u0[j])
        idx = np.arange(nx)
        assert np.array_equal(out[j], 0.5 * (F[(idx - S) % len(F)] + F[(idx + S) % len(F)]))


def test_fp32_rounding_of_the_two_forms():
    """Why FP32 runs use the increment form: with small steps the per-step change falls far
    below one ulp of u, and the standard form (which recomputes the velocity from two rounded
    levels) drifts, while the increment form stays at the FP32 bar.  Point singularity on 257^2,
    CFL 0.02, 2000 steps, against the FP64 oracle."""
    n, S = 257, 2000
    g = oracle.grid(n, n)
    depth = dict(background=0.5, eps=4 / (n - 1), mollifier=0, sings=[(2, 1, 0.01, 0.5, 0.5)])
    hx, hy, ext = oracle.make_depth(g, depth)
    u0 = inputs.gaussian_hump(n, n, None, 0.3, 0.5, 0.05)
    tau = 0.02 * g.dx / math.sqrt(max(ext[1], ext[3]))
    ref = oracle.forward(g, tau, hx, hy, u0, None, S, want_energy=False)["u"]
    e_std = relerr(oracle.forward_f32(g, tau, hx, hy, u0, None, S, False), ref)
    e_inc = relerr(oracle.forward_f32(g, tau, hx, hy, u0, None, S, True), ref)
    assert e_inc <= 1e-5, e_inc
    assert e_std >= 100 * e_inc, (e_std, e_inc)
