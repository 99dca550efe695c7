"""FP64 CPU oracle for the regularised 2D tsunami wave equation (leapfrog).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never stands in for it.

The arithmetic lives in ``tsu_oracle.c`` (plain C, FP64, no fused multiply-add);
this module compiles it with gcc on first use and wraps it with numpy arrays.
Paper passages followed (arXiv:2005.11931):

* Sec. 2, eq. (2.1): ``u_tt - sum_j d_j(h_j d_j u) = 0`` with vector depth.
* Sec. 2.1: regularisation ``h_eps = h * psi_eps``, ``psi_eps = eps^-1 psi(x/eps)``.  That
  normalisation has unit mass only on the line; the 2D point mollifier is scaled by ``eps^-2``
  so that it keeps unit mass in the plane.
* Sec. 3.1: the Friedrichs bump ``c exp(1/(x^2-1))`` with ``c ~ 2.2523``; delta and
  delta^2 singularities ``phi_eps`` and ``phi_eps^2``; the step depth h0.
* Sec. 3.3: the 2D box with zero Dirichlet edges and the grid omega.
* Theorem 2.1, identity (CL-01): conservation of ``||u_t||^2 + sum ||h_j^1/2 d_j u||^2``,
  whose leapfrog analogue is ``energy``.
* Sec. 3.3: the implicit scheme solved line by line with tridiagonal systems, read as the
  factorized scheme ``(I - sigma B_x)(I - sigma B_y) w = B u`` (``implicit_forward``).

Arrays are float64, shape ``(ny, ld)`` with ``ld >= nx``, row-major (x fastest).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsu_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libtsu_oracle.so")
_lock = threading.Lock()
_lib = None

# singularity kinds and mollifiers (the oracle's own numbering)
LINE_X, LINE_Y, POINT, STEP_X, STEP_Y = 0, 1, 2, 3, 4
GAUSS, FRIEDRICHS = 0, 1


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("ld", C.c_int64),
                ("dx", C.c_double), ("dy", C.c_double)]


class _Sing(C.Structure):
    _fields_ = [("kind", C.c_int32), ("power", C.c_int32), ("amp", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double)]


class _Depth(C.Structure):
    _fields_ = [("background", C.c_double), ("eps", C.c_double), ("mollifier", C.c_int32),
                ("nsing", C.c_int32), ("sing", C.POINTER(_Sing))]


def build(force: bool = False) -> str:
    """Compile ``tsu_oracle.c`` into ``_build/libtsu_oracle.so`` (gcc, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = C.CDLL(path)
        d = C.POINTER(C.c_double)
        g = C.POINTER(_Grid)
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_set_threads.restype = C.c_int
        lib.orc_friedrichs_c1.restype = C.c_double
        lib.orc_friedrichs_c2.restype = C.c_double
        lib.orc_make_depth.argtypes = [g, C.POINTER(_Depth), d, d, d]
        lib.orc_make_depth.restype = C.c_int
        lib.orc_forward_f32.argtypes = [g, C.c_double, d, d, d, d, C.c_int64, C.c_int, d]
        lib.orc_forward_f32.restype = C.c_int
        lib.orc_depth_deps.argtypes = [g, C.POINTER(_Depth), d, d]
        lib.orc_depth_deps.restype = C.c_int
        lib.orc_apply_B.argtypes = [g, C.c_double, C.c_double, d, d, d, d]
        lib.orc_init.argtypes = [g, C.c_double, d, d, d, d, d, d]
        lib.orc_step.argtypes = [g, C.c_double, d, d, d, d]
        lib.orc_energy.argtypes = [g, C.c_double, d, d, d, d]
        lib.orc_energy.restype = C.c_double
        lib.orc_forward.argtypes = [g, C.c_double, d, d, d, d, C.c_int64, d, C.c_int32,
                                    C.POINTER(C.c_int64), d, d, d]
        lib.orc_forward.restype = C.c_int
        lib.orc_adjoint.argtypes = [g, C.c_double, d, d, d, d, C.c_int64, C.c_int32,
                                    C.POINTER(C.c_int64), d, d, d, d, d]
        lib.orc_adjoint.restype = C.c_int
        lib.orc_implicit_forward.argtypes = [g, C.c_double, C.c_double, d, d, d, d, C.c_int64, d, d]
        lib.orc_implicit_forward.restype = C.c_int
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def grid(nx: int, ny: int, ld: int | None = None) -> _Grid:
    """Unit box [0,1]^2 with nx x ny nodes including the boundary."""
    return _Grid(nx, ny, ld or nx, 1.0 / (nx - 1), 1.0 / (ny - 1))


def _field(g, a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (g.ny, g.ld), (a.shape, (g.ny, g.ld))
    return a


def set_threads(n: int) -> int:
    """Number of OpenMP threads the oracle uses (returns the effective count)."""
    return int(_load().orc_set_threads(int(n)))


def friedrichs_constants() -> tuple[float, float]:
    """(c1, c2): normalisers of the 1D and 2D Friedrichs bumps (Sec. 3.1)."""
    lib = _load()
    return float(lib.orc_friedrichs_c1()), float(lib.orc_friedrichs_c2())


def make_depth(g: _Grid, depth: dict):
    """Face-sampled mollified depth.  ``depth`` = {background, eps, mollifier,
    sings: [(kind, power, amp, cx, cy), ...]}.  Returns (hx, hy, ext) with
    ext = [min hx, max hx, min hy, max hy]."""
    lib = _load()
    sings = depth.get("sings", [])
    arr = (_Sing * max(1, len(sings)))(*[_Sing(*s) for s in sings])
    d = _Depth(float(depth["background"]), float(depth["eps"]), int(depth.get("mollifier", GAUSS)),
               len(sings), C.cast(arr, C.POINTER(_Sing)))
    hx = np.zeros((g.ny, g.ld))
    hy = np.zeros((g.ny, g.ld))
    ext = np.zeros(4)
    rc = lib.orc_make_depth(C.byref(g), C.byref(d), _p(hx), _p(hy), _p(ext))
    if rc != 0:
        raise ValueError("oracle make_depth: bad arguments")
    return hx, hy, ext


def forward_f32(g, tau, hx, hy, u0, u1, steps: int, increment: bool):
    """The start and ``steps-1`` leapfrog steps in FP32 arithmetic (no fused multiply-add), in the
    standard or the increment form; returns u^S widened to FP64.  Shows the FP32 rounding of each
    form without any GPU code."""
    out = np.zeros((g.ny, g.ld))
    rc = _load().orc_forward_f32(C.byref(g), tau, _p(_field(g, hx)), _p(_field(g, hy)), _p(_field(g, u0)),
                                 _p(_field(g, u1)), int(steps), int(bool(increment)), _p(out))
    if rc != 0:
        raise ValueError("oracle forward_f32: bad arguments")
    return out


def depth_deps(g: _Grid, depth: dict):
    """d h_eps / d eps at the faces (same layout as make_depth's hx, hy): the derivative of the
    regularised depth with respect to the regularisation width (Sec. 2.1).  Returns (dhx, dhy)."""
    lib = _load()
    sings = depth.get("sings", [])
    arr = (_Sing * max(1, len(sings)))(*[_Sing(*s) for s in sings])
    d = _Depth(float(depth["background"]), float(depth["eps"]), int(depth.get("mollifier", GAUSS)),
               len(sings), C.cast(arr, C.POINTER(_Sing)))
    dhx = np.zeros((g.ny, g.ld))
    dhy = np.zeros((g.ny, g.ld))
    if lib.orc_depth_deps(C.byref(g), C.byref(d), _p(dhx), _p(dhy)) != 0:
        raise ValueError("oracle depth_deps: bad arguments")
    return dhx, dhy


def coefs(g: _Grid, tau: float) -> tuple[float, float]:
    return tau * tau / (g.dx * g.dx), tau * tau / (g.dy * g.dy)


def apply_B(g, tau, hx, hy, u):
    """B u = tau^2 L_h u on interior nodes (0 on the boundary)."""
    out = np.zeros((g.ny, g.ld))
    cx, cy = coefs(g, tau)
    _load().orc_apply_B(C.byref(g), cx, cy, _p(_field(g, hx)), _p(_field(g, hy)),
                        _p(_field(g, u)), _p(out))
    return out


def init(g, tau, hx, hy, u0, u1=None):
    """Taylor start: returns (u^0 with zero boundary, u^1)."""
    up = np.zeros((g.ny, g.ld))
    uc = np.zeros((g.ny, g.ld))
    _load().orc_init(C.byref(g), tau, _p(_field(g, hx)), _p(_field(g, hy)), _p(_field(g, u0)),
                     _p(_field(g, u1)), _p(up), _p(uc))
    return up, uc


def step(g, tau, hx, hy, u_prev, u_cur):
    """One leapfrog step; returns u^{n+1} (inputs are not modified)."""
    out = np.array(_field(g, u_prev), copy=True)
    _load().orc_step(C.byref(g), tau, _p(_field(g, hx)), _p(_field(g, hy)), _p(out),
                     _p(_field(g, u_cur)))
    return out


def energy(g, tau, hx, hy, u_n, u_n1) -> float:
    """Discrete energy E^{n+1/2} of the pair (u^n, u^{n+1})."""
    return float(_load().orc_energy(C.byref(g), tau, _p(_field(g, hx)), _p(_field(g, hy)),
                                    _p(_field(g, u_n)), _p(_field(g, u_n1))))


def forward(g, tau, hx, hy, u0, u1, steps: int, want_energy=True, rec_idx=None):
    """Taylor start then ``steps-1`` leapfrog steps (``steps`` counts the start).

    Returns dict(u_prev=u^{S-1}, u=u^S, energy=[E^{1/2}..E^{S-1/2}],
    traces=[S][nrec] with traces[n-1] = u^n at the receivers)."""
    lib = _load()
    up = np.zeros((g.ny, g.ld))
    uc = np.zeros((g.ny, g.ld))
    en = np.zeros(steps) if want_energy else None
    if rec_idx is not None:
        ri = np.ascontiguousarray(rec_idx, dtype=np.int64)
        tr = np.zeros((steps, len(ri)))
        rp = ri.ctypes.data_as(C.POINTER(C.c_int64))
        nrec = len(ri)
    else:
        tr, rp, nrec = None, None, 0
    rc = lib.orc_forward(C.byref(g), tau, _p(_field(g, hx)), _p(_field(g, hy)), _p(_field(g, u0)),
                         _p(_field(g, u1)), int(steps), _p(en), nrec, rp, _p(tr), _p(up), _p(uc))
    if rc != 0:
        raise ValueError("oracle forward: bad arguments")
    return dict(u_prev=up, u=uc, energy=en, traces=tr)


def adjoint(g, tau, hx, hy, u0, u1, steps: int, rec_idx, dtraces):
    """Discrete adjoint of ``forward`` for J with dJ/dtraces = ``dtraces`` [S][nrec].

    Returns dict(g_hx, g_hy, g_u0, g_u1)."""
    lib = _load()
    ri = np.ascontiguousarray(rec_idx, dtype=np.int64)
    dt = np.ascontiguousarray(dtraces, dtype=np.float64)
    assert dt.shape == (steps, len(ri))
    out = {k: np.zeros((g.ny, g.ld)) for k in ("g_hx", "g_hy", "g_u0", "g_u1")}
    rc = lib.orc_adjoint(C.byref(g), tau, _p(_field(g, hx)), _p(_field(g, hy)), _p(_field(g, u0)),
                         _p(_field(g, u1)), int(steps), len(ri), ri.ctypes.data_as(C.POINTER(C.c_int64)),
                         _p(dt), _p(out["g_hx"]), _p(out["g_hy"]), _p(out["g_u0"]), _p(out["g_u1"]))
    if rc != 0:
        raise ValueError(f"oracle adjoint failed ({rc})")
    return out


def implicit_forward(g, tau, sigma, hx, hy, u0, u1, steps: int):
    """The implicit comparator (Sec. 3.3, read as the factorized scheme with weight ``sigma``):
    ``(I - sigma B_x)(I - sigma B_y) w^n = B u^n``, ``v^{n+1} = v^n + w^n``, ``u^{n+1} = u^n +
    v^{n+1}``, started by ``v^1 = tau u1 + w^0 / 2``.  Every factor is solved line by line with
    Thomas elimination.  Returns (u^S, v^S) after the start and ``steps - 1`` steps."""
    u = np.zeros((g.ny, g.ld))
    v = np.zeros((g.ny, g.ld))
    rc = _load().orc_implicit_forward(C.byref(g), float(tau), float(sigma), _p(_field(g, hx)), _p(_field(g, hy)),
                                      _p(_field(g, u0)), _p(_field(g, u1)), int(steps), _p(u), _p(v))
    if rc != 0:
        raise ValueError(f"oracle implicit_forward failed ({rc})")
    return u, v
