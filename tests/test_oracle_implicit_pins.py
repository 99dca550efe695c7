"""Pins of the oracle's implicit comparator (Sec. 3.3: an implicit scheme solved along grid lines,
read as the factorized scheme (I - s B_x)(I - s B_y) w^n = B u^n in increment form).

No GPU.  Each check compares the oracle with something other than itself:
- a dense linear solve of the same scheme, assembled here from the face depths;
- the closed-form evolution of a separable mode, at time steps far above the explicit limit;
- the explicit leapfrog oracle (s = 0 reduces the scheme to it);
- the scheme's conserved energy for constant depth;
- mirror symmetry;
- second-order convergence in time.

A slip in the line solver (a face index off by one, the factors in the wrong order, a
sub-diagonal with the wrong sign, a dropped 1/2 in the start) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_11931_gb300 import inputs


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dense_operators(nx, ny, cx, cy, hx, hy):
    """B_x and B_y on the interior nodes (p = (j-1)(nx-2) + (i-1)), assembled from the face
    depths: (B_x u)_ij = cx [hx_ij (u_i+1,j - u_ij) - hx_i-1,j (u_ij - u_i-1,j)], likewise B_y."""
    m = (nx - 2) * (ny - 2)
    Bx = np.zeros((m, m))
    By = np.zeros((m, m))
    p = lambda i, j: (j - 1) * (nx - 2) + (i - 1)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            q = p(i, j)
            Bx[q, q] = -cx * (hx[j, i - 1] + hx[j, i])
            if i > 1:
                Bx[q, p(i - 1, j)] = cx * hx[j, i - 1]
            if i < nx - 2:
                Bx[q, p(i + 1, j)] = cx * hx[j, i]
            By[q, q] = -cy * (hy[j - 1, i] + hy[j, i])
            if j > 1:
                By[q, p(i, j - 1)] = cy * hy[j - 1, i]
            if j < ny - 2:
                By[q, p(i, j + 1)] = cy * hy[j, i]
    return Bx, By


@pytest.mark.parametrize("nx,ny,S,sigma,cfl", [(7, 6, 6, 0.25, 3.0), (9, 5, 11, 0.5, 8.0), (3, 8, 4, 0.25, 2.0)])
def test_implicit_matches_dense_solve(nx, ny, S, sigma, cfl):
    """Random positive faces (the factors do not commute), random data: every step solved with a
    dense LU of A = (I - s B_x)(I - s B_y)."""
    rng = np.random.default_rng(7)
    g = oracle.grid(nx, ny)
    hx = rng.uniform(0.5, 2.0, (ny, nx))
    hy = rng.uniform(0.5, 2.0, (ny, nx))
    tau = cfl * min(g.dx, g.dy) / math.sqrt(2.0)
    cx, cy = tau * tau / g.dx ** 2, tau * tau / g.dy ** 2
    u0 = np.zeros((ny, nx))
    u1 = np.zeros((ny, nx))
    u0[1:-1, 1:-1] = rng.standard_normal((ny - 2, nx - 2))
    u1[1:-1, 1:-1] = rng.standard_normal((ny - 2, nx - 2))
    Bx, By = dense_operators(nx, ny, cx, cy, hx, hy)
    I = np.eye(Bx.shape[0])
    A = (I - sigma * Bx) @ (I - sigma * By)
    B = Bx + By
    u = u0[1:-1, 1:-1].reshape(-1)
    v = tau * u1[1:-1, 1:-1].reshape(-1) + 0.5 * np.linalg.solve(A, B @ u)
    u = u + v
    for _ in range(S - 1):
        v = v + np.linalg.solve(A, B @ u)
        u = u + v
    got_u, got_v = oracle.implicit_forward(g, tau, sigma, hx, hy, u0, u1, S)
    assert relerr(got_u[1:-1, 1:-1].reshape(-1), u) < 1e-12
    assert relerr(got_v[1:-1, 1:-1].reshape(-1), v) < 1e-12
    assert not got_u[0].any() and not got_u[-1].any() and not got_u[:, 0].any() and not got_u[:, -1].any()


def test_dense_check_sees_swapped_factors():
    """Sanity of the dense check: with non-commuting factors, (I - s B_y)(I - s B_x) differs
    from the oracle's (I - s B_x)(I - s B_y) by far more than round-off."""
    nx, ny, S, sigma = 7, 6, 6, 0.25
    rng = np.random.default_rng(7)
    g = oracle.grid(nx, ny)
    hx = rng.uniform(0.5, 2.0, (ny, nx))
    hy = rng.uniform(0.5, 2.0, (ny, nx))
    tau = 3.0 * min(g.dx, g.dy) / math.sqrt(2.0)
    cx, cy = tau * tau / g.dx ** 2, tau * tau / g.dy ** 2
    u0 = np.zeros((ny, nx))
    u0[1:-1, 1:-1] = rng.standard_normal((ny - 2, nx - 2))
    Bx, By = dense_operators(nx, ny, cx, cy, hx, hy)
    I = np.eye(Bx.shape[0])
    A_swapped = (I - sigma * By) @ (I - sigma * Bx)
    B = Bx + By
    u = u0[1:-1, 1:-1].reshape(-1)
    v = 0.5 * np.linalg.solve(A_swapped, B @ u)
    u = u + v
    for _ in range(S - 1):
        v = v + np.linalg.solve(A_swapped, B @ u)
        u = u + v
    got_u, _ = oracle.implicit_forward(g, tau, sigma, hx, hy, u0, None, S)
    assert relerr(got_u[1:-1, 1:-1].reshape(-1), u) > 1e-6


@pytest.mark.parametrize("nx,ny,k,l,S,h0,vel,cfl", [
    (33, 33, 1, 1, 200, 1.0, 0.0, 3.0),
    (41, 29, 2, 5, 300, 0.7, 1.3, 20.0),
    (17, 65, 7, 1, 120, 1.0, -0.4, 0.5),
])
def test_implicit_separable_mode_exact(nx, ny, k, l, S, h0, vel, cfl):
    """Constant depth h0: phi = sin(k pi x) sin(l pi y) has B_x phi = -lx phi, B_y phi = -ly phi,
    lx = 4 cx h0 sin^2(k pi dx/2).  The scheme then gives u^n = a_n phi with
    a_n = cos(n w) + tau vel sin(n w)/sin(w), cos(w) = 1 - (lx + ly) / (2 (1 + s lx)(1 + s ly)),
    start included, at any Courant number when s = 1/4 (here up to 20)."""
    sigma = 0.25
    g = oracle.grid(nx, ny)
    hx, hy, _ = oracle.make_depth(g, dict(background=h0, eps=0.1, sings=[]))
    tau = cfl * min(g.dx, g.dy) / math.sqrt(h0)
    phi = inputs.separable_mode(nx, ny, None, k, l)
    cx, cy = tau * tau / g.dx ** 2, tau * tau / g.dy ** 2
    lx = 4 * cx * h0 * math.sin(k * math.pi * g.dx / 2) ** 2
    ly = 4 * cy * h0 * math.sin(l * math.pi * g.dy / 2) ** 2
    w = math.acos(1 - (lx + ly) / (2 * (1 + sigma * lx) * (1 + sigma * ly)))
    a = lambda n: math.cos(n * w) + tau * vel * math.sin(n * w) / math.sin(w)
    u, v = oracle.implicit_forward(g, tau, sigma, hx, hy, phi, vel * phi, S)
    assert np.max(np.abs(u - a(S) * phi)) < 1e-11 * max(1.0, abs(a(S)))
    assert np.max(np.abs(v - (a(S) - a(S - 1)) * phi)) < 1e-11 * max(1.0, abs(a(S)))


def test_implicit_with_zero_weight_is_the_explicit_scheme():
    """s = 0: A = I and the scheme is the explicit leapfrog (the increment form of it)."""
    n = 61
    g = oracle.grid(n, n - 10)
    depth = dict(background=0.8, eps=0.05, sings=[(inputs.POINT, 1, 0.004, 0.4, 0.45),
                                                  (inputs.LINE_X, 1, 0.6, 0.62, 0.5)])
    hx, hy, ext = oracle.make_depth(g, depth)
    tau = 0.4 * min(g.dx, g.dy) / math.sqrt(max(ext[1], ext[3]))
    u0 = inputs.gaussian_hump(g.nx, g.ny, None, 0.3, 0.5, 0.08)
    u1 = 0.5 * inputs.gaussian_hump(g.nx, g.ny, None, 0.5, 0.4, 0.1)
    ref = oracle.forward(g, tau, hx, hy, u0, u1, 300, want_energy=False)
    u, v = oracle.implicit_forward(g, tau, 0.0, hx, hy, u0, u1, 300)
    assert relerr(u, ref["u"]) < 1e-12
    assert relerr(v, ref["u"] - ref["u_prev"]) < 1e-10


def _energy(g, tau, sigma, hx, hy, u_n, u_n1):
    """E^{n+1/2} = <A v, v> - <B u^{n+1}, u^n> with v = u^{n+1} - u^n: conserved exactly by the
    factorized scheme when A is symmetric (constant depth)."""
    cx, cy = tau * tau / g.dx ** 2, tau * tau / g.dy ** 2

    def bx(f):
        out = np.zeros_like(f)
        out[1:-1, 1:-1] = cx * (hx[1:-1, 1:-1] * (f[1:-1, 2:] - f[1:-1, 1:-1])
                                - hx[1:-1, :-2] * (f[1:-1, 1:-1] - f[1:-1, :-2]))
        return out

    def by(f):
        out = np.zeros_like(f)
        out[1:-1, 1:-1] = cy * (hy[1:-1, 1:-1] * (f[2:, 1:-1] - f[1:-1, 1:-1])
                                - hy[:-2, 1:-1] * (f[1:-1, 1:-1] - f[:-2, 1:-1]))
        return out

    v = u_n1 - u_n
    Av = v - sigma * bx(v) - sigma * by(v) + sigma * sigma * bx(by(v))
    return float(np.sum(Av * v) - np.sum((bx(u_n1) + by(u_n1)) * u_n))


def test_implicit_energy_conserved_constant_depth():
    """Constant depth, Courant number 5 (five times beyond the explicit limit), nonzero initial
    velocity: the factorized scheme's energy stays constant to round-off."""
    n, S, sigma, h0 = 49, 400, 0.25, 1.3
    g = oracle.grid(n, n - 8)
    hx, hy, _ = oracle.make_depth(g, dict(background=h0, eps=0.1, sings=[]))
    tau = 5.0 * min(g.dx, g.dy) / math.sqrt(h0)
    u0 = inputs.gaussian_hump(g.nx, g.ny, None, 0.3, 0.5, 0.08)
    u1 = 0.5 * inputs.gaussian_hump(g.nx, g.ny, None, 0.5, 0.4, 0.1)
    u_1, _ = oracle.implicit_forward(g, tau, sigma, hx, hy, u0, u1, 1)
    u_a, _ = oracle.implicit_forward(g, tau, sigma, hx, hy, u0, u1, S - 1)
    u_b, v_b = oracle.implicit_forward(g, tau, sigma, hx, hy, u0, u1, S)
    assert relerr(u_b - v_b, u_a) < 1e-13
    u0z = u0.copy()
    u0z[0], u0z[-1], u0z[:, 0], u0z[:, -1] = 0, 0, 0, 0
    e0 = _energy(g, tau, sigma, hx, hy, u0z, u_1)
    e1 = _energy(g, tau, sigma, hx, hy, u_a, u_b)
    assert e0 > 0
    assert abs(e1 - e0) / e0 < 1e-11, (e0, e1)


def test_implicit_mirror_symmetry():
    """Depth independent of y and a hump centred at y = 0.5: the solution is symmetric under
    y -> 1 - y (to round-off: the eliminations run in one direction)."""
    n = 101
    g = oracle.grid(n, n)
    depth = inputs.paper_case1_2d(n=n)["problem"].depth
    hx, hy, ext = oracle.make_depth(g, depth)
    tau = 4.0 * g.dx / math.sqrt(max(ext[1], ext[3]))
    u0 = inputs.gaussian_hump(n, n, None, 0.4, 0.5, 0.05)
    u, _ = oracle.implicit_forward(g, tau, 0.25, hx, hy, u0, None, 80)
    assert np.abs(u).max() > 0.01
    assert np.max(np.abs(u - u[::-1, :])) < 1e-13 * np.abs(u).max()


def test_implicit_second_order_in_time():
    """At a fixed time and grid, the scheme converges to the semi-discrete solution at second
    order in tau (reference: the explicit leapfrog at a 16 times smaller step)."""
    n = 65
    g = oracle.grid(n, n)
    depth = dict(background=1.0, eps=0.06, sings=[(inputs.LINE_X, 1, 1.0, 0.55, 0.5)])
    hx, hy, ext = oracle.make_depth(g, depth)
    u0 = inputs.gaussian_hump(n, n, None, 0.35, 0.5, 0.08)
    T = 0.3
    base = 2.0 * g.dx / math.sqrt(max(ext[1], ext[3]))  # Courant number 2 at the coarsest step
    S0 = int(math.ceil(T / base))
    tau0 = T / S0
    ref = oracle.forward(g, tau0 / 64, hx, hy, u0, None, 64 * S0, want_energy=False)["u"]
    errs = []
    for m in (1, 2, 4):
        u, _ = oracle.implicit_forward(g, tau0 / m, 0.25, hx, hy, u0, None, m * S0)
        errs.append(relerr(u, ref))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
