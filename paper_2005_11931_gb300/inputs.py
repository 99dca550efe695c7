"""Seeded synthetic inputs for the regularised 2D tsunami workloads.

This module is shared by the CUDA path and by the oracle's tests.  It holds
only *inputs*: problem descriptions (grid sizes, singularity placements,
mollifier width, step counts), initial displacements sampled at the nodes,
receiver positions and random directions.  It contains none of the method's
arithmetic (no mollifier, no face sampling, no stencil, no time step).

The workloads restate the paper's 2D experiments (Sec. 3.3: a Gaussian initial
hump, zero initial velocity, zero Dirichlet edges, a depth with a line or
point singularity regularised at width eps) on the unit box [0,1]^2.
The paper measures on no public dataset; everything here is analytic or drawn
from ``numpy.random.default_rng(2005_11931)``.

Depth descriptors are plain dicts:
``{"background": b, "eps": e, "mollifier": 0|1, "sings": [(kind, power, amp, cx, cy), ...]}``
with kind 0 = line varying in x (delta(x - cx)), 1 = line varying in y,
2 = point, 3 = step in x (amp for x < cx), 4 = step in y; mollifier 0 = Gaussian,
1 = Friedrichs bump.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 2005_11931
LINE_X, LINE_Y, POINT, STEP_X, STEP_Y = 0, 1, 2, 3, 4
GAUSS, FRIEDRICHS = 0, 1
CFL = 0.4  # tau = CFL * dx / sqrt(max h) in every workload


def padded_ld(nx: int, align: int = 32) -> int:
    """Row pitch in elements: nx rounded up so that every row starts 128-B aligned."""
    return (nx + align - 1) // align * align


def node_offsets(n: int, c: float) -> np.ndarray:
    """Coordinates x_i - c of the n nodes of [0,1] (spacing 1/(n-1)).

    Written as (i - c (n-1)) / (n-1) so that data centred on a node or on a
    half node is mirror symmetric bit for bit."""
    i = np.arange(n, dtype=np.float64)
    return (i - c * (n - 1)) / (n - 1)


def gaussian_hump(nx: int, ny: int, ld: int | None, x0: float, y0: float, width: float,
                  amplitude: float = 1.0, dtype=np.float64) -> np.ndarray:
    """u0(x, y) = amplitude * exp(-((x-x0)^2 + (y-y0)^2) / width^2) at the nodes,
    shape (ny, ld) with zero padding columns."""
    ld = ld or nx
    dxo = node_offsets(nx, x0)
    dyo = node_offsets(ny, y0)
    r2 = dyo[:, None] ** 2 + dxo[None, :] ** 2
    out = np.zeros((ny, ld), dtype=np.float64)
    out[:, :nx] = amplitude * np.exp(-r2 / (width * width))
    return out.astype(dtype)


def separable_mode(nx: int, ny: int, ld: int | None, k: int, l: int, dtype=np.float64) -> np.ndarray:
    """sin(k pi x) sin(l pi y) at the nodes (zero on the boundary up to rounding)."""
    ld = ld or nx
    x = np.arange(nx) / (nx - 1)
    y = np.arange(ny) / (ny - 1)
    out = np.zeros((ny, ld))
    out[:, :nx] = np.sin(l * np.pi * y)[:, None] * np.sin(k * np.pi * x)[None, :]
    out[0, :] = 0
    out[-1, :] = 0
    out[:, 0] = 0
    out[:, nx - 1] = 0
    return out.astype(dtype)


def random_field(nx: int, ny: int, ld: int | None, rng: np.random.Generator, dtype=np.float64,
                 zero_boundary: bool = True) -> np.ndarray:
    ld = ld or nx
    out = np.zeros((ny, ld))
    out[:, :nx] = rng.standard_normal((ny, nx))
    if zero_boundary:
        out[0, :] = 0
        out[-1, :] = 0
        out[:, 0] = 0
        out[:, nx - 1] = 0
    return out.astype(dtype)


def receivers_on_row(n: int, y: float, count: int, rng: np.random.Generator) -> np.ndarray:
    """``count`` receiver nodes (i, j) on the row nearest y, i drawn without replacement from [1, n-2]."""
    j = int(round(y * (n - 1)))
    i = np.sort(rng.choice(np.arange(1, n - 1), size=count, replace=False))
    return np.stack([i, np.full_like(i, j)], axis=1).astype(np.int64)


def flat_index(ij: np.ndarray, ld: int) -> np.ndarray:
    return (ij[:, 1].astype(np.int64) * ld + ij[:, 0].astype(np.int64))


@dataclass
class Problem:
    """One forward problem on the unit box."""
    name: str
    n: int                       # nodes per side, boundary included
    depth: dict
    u0: tuple                    # (x0, y0, width, amplitude)
    steps: int                   # S: final state u^S (the Taylor start is step 1)
    dtype: str = "f32"
    extra: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return 1.0 / (self.n - 1)

    @property
    def lups(self) -> int:
        """Interior lattice-point updates of the whole run (S steps)."""
        return (self.n - 2) * (self.n - 2) * self.steps

    def initial(self, ld: int | None = None, dtype=np.float64) -> np.ndarray:
        x0, y0, w, a = self.u0
        return gaussian_hump(self.n, self.n, ld, x0, y0, w, a, dtype)


def line_fp64_201() -> Problem:
    """201^2 FP64 parity case: depth 1 + phi_eps(x - 0.5), eps = 0.02, hump of width
    0.05 at (0.25, 0.5), 1000 steps, energy every step."""
    return Problem("line_fp64_201", 201,
                   dict(background=1.0, eps=0.02, mollifier=GAUSS, sings=[(LINE_X, 1, 1.0, 0.5, 0.5)]),
                   (0.25, 0.5, 0.05, 1.0), 1000, "f64")


def point_fp32(n: int = 8192, steps: int = 5000) -> Problem:
    """Point singularity 0.5 + 0.01 phi_eps(|r - (0.5,0.5)|), eps = 4 dx, hump of width
    0.02 at (0.3, 0.5).  Default: 8192^2, 5000 steps, FP32 fields."""
    dx = 1.0 / (n - 1)
    return Problem(f"point_fp32_{n}", n,
                   dict(background=0.5, eps=4 * dx, mollifier=GAUSS, sings=[(POINT, 1, 0.01, 0.5, 0.5)]),
                   (0.3, 0.5, 0.02, 1.0), steps, "f32")


def crossing_lines_fp32(n: int = 16384, steps: int = 20000) -> Problem:
    """Crossing lines 1 + phi_eps(x-0.5) + phi_eps(y-0.5), eps = 8 dx, hump of width
    0.01 at (0.25, 0.25).  Default: 16384^2, 20000 steps, FP32 fields."""
    dx = 1.0 / (n - 1)
    return Problem(f"crossing_lines_fp32_{n}", n,
                   dict(background=1.0, eps=8 * dx, mollifier=GAUSS,
                        sings=[(LINE_X, 1, 1.0, 0.5, 0.5), (LINE_Y, 1, 1.0, 0.5, 0.5)]),
                   (0.25, 0.25, 0.01, 1.0), steps, "f32")


def adjoint_case(n: int = 2048, steps: int = 4000, nrec: int = 128, eps: float = 0.01,
                 eps_obs: float = 0.012) -> dict:
    """Receiver-misfit case: depth 1 + 0.5 phi_eps(x - 0.5), hump of width 0.03 at
    (0.42, 0.70), ``nrec`` receivers on the row y = 0.8, observations from eps_obs."""
    rng = np.random.default_rng(SEED)
    rec = receivers_on_row(n, 0.8, nrec, rng)
    mk = lambda e: dict(background=1.0, eps=e, mollifier=GAUSS, sings=[(LINE_X, 1, 0.5, 0.5, 0.5)])
    prob = Problem(f"adjoint_{n}", n, mk(eps), (0.42, 0.70, 0.03, 1.0), steps, "f32")
    return dict(problem=prob, depth_obs=mk(eps_obs), receivers=rec, ckpt_every=64, rng=rng)


def batched_family(steps: int = 2000, count_eps: int = 16,
                   sizes=(512, 768, 1024, 1536, 2048)) -> list[Problem]:
    """The eps-family: ``count_eps`` widths log-spaced in [1/512, 1/16] times four
    singularity types (line in x, line in y, point, line + point) on background 1,
    per-problem size drawn from ``sizes``, hump of width 0.03 at a seeded centre in
    [0.2, 0.8]^2."""
    rng = np.random.default_rng(SEED)
    eps_list = np.logspace(math.log10(1 / 512), math.log10(1 / 16), count_eps)
    types = {
        "line_x": [(LINE_X, 1, 1.0, 0.5, 0.5)],
        "line_y": [(LINE_Y, 1, 1.0, 0.5, 0.5)],
        "point": [(POINT, 1, 0.01, 0.5, 0.5)],
        "line_point": [(LINE_X, 1, 1.0, 0.5, 0.5), (POINT, 1, 0.01, 0.5, 0.5)],
    }
    probs = []
    for e_i, eps in enumerate(eps_list):
        for tname, sings in types.items():
            n = int(rng.choice(sizes))
            x0, y0 = rng.uniform(0.2, 0.8, size=2)
            probs.append(Problem(f"fam_{e_i:02d}_{tname}_{n}", n,
                                 dict(background=1.0, eps=float(eps), mollifier=GAUSS, sings=sings),
                                 (float(x0), float(y0), 0.03, 1.0), steps, "f32",
                                 extra=dict(eps_index=e_i, kind=tname)))
    return probs


def paper_case1_2d(n: int = 513, eps: float = 0.8, steps: int = 200) -> dict:
    """The paper's own 2D workload (Sec. 3.3) rescaled from [0,100]^2 to the unit box:
    depth h0(x) = 100 for x < 75, 10 after (a step at x = 0.75), mollified at eps/100;
    u0 = 50 exp(-((x-40)^2 + (y-50)^2)/8) -> width sqrt(8)/100 at (0.40, 0.50).
    Time is rescaled by 1/100 as well (the wave speed sqrt(h) is unchanged)."""
    depth = dict(background=10.0, eps=eps / 100.0, mollifier=FRIEDRICHS,
                 sings=[(STEP_X, 1, 90.0, 0.75, 0.5)])
    return dict(problem=Problem(f"paper_case1_{n}", n, depth, (0.40, 0.50, math.sqrt(8) / 100, 50.0),
                                steps, "f64"))


def paper_table1(n: int, steps: int = 100, dtype: str = "f64") -> Problem:
    """The paper's GPU timing runs (Sec. 4, Table 1): the 2D Case 1 problem of paper_case1_2d on
    n x n nodes (the paper's 256 .. 4096), dt = 0.05 in paper units, T = 5.0, so 100 steps.  In
    the unit box the step is tau = 0.05 / 100 (time rescales with length); its Courant number
    tau sqrt(100) / dx grows from 1.3 (256) to 20 (4096), beyond any explicit scheme, which is
    why the paper's scheme is implicit."""
    p = paper_case1_2d(n=n, steps=steps)["problem"]
    return Problem(f"paper_table1_{n}", n, p.depth, p.u0, steps, dtype, extra=dict(tau=0.05 / 100.0))


def random_directions(shape, count: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal((count,) + tuple(shape))
