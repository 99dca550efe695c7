"""Thin Python binding of libtsu (include/tsu.h).

Argument marshalling only: every step of the computation runs in the CUDA kernels of
``libtsu.so``.  PyTorch supplies device memory and streams.  The functions carry the C names
(``tsu_make_depth``, ``tsu_init``, ``tsu_step_n`` ...); ``Simulation`` bundles the buffers of
one forward problem.  If the library has not been built, ``load()`` raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsu.so")

TSU_OK, TSU_EINVAL, TSU_ECFL, TSU_ENONPOS, TSU_ENOMEM, TSU_ECUDA, TSU_ETIMEOUT = range(7)
TSU_F32, TSU_F64 = 0, 1
TSU_FORM_STANDARD, TSU_FORM_INCREMENT = 0, 1
TSU_LINE_X, TSU_LINE_Y, TSU_POINT, TSU_STEP_X, TSU_STEP_Y = range(5)
TSU_GAUSS, TSU_FRIEDRICHS = 0, 1
_NAMES = {0: "TSU_OK", 1: "TSU_EINVAL", 2: "TSU_ECFL", 3: "TSU_ENONPOS", 4: "TSU_ENOMEM", 5: "TSU_ECUDA",
          6: "TSU_ETIMEOUT"}

DTYPES = {TSU_F32: torch.float32, TSU_F64: torch.float64, "f32": torch.float32, "f64": torch.float64}


def dtype_code(dt) -> int:
    if dt in (TSU_F32, "f32", torch.float32, np.float32):
        return TSU_F32
    if dt in (TSU_F64, "f64", torch.float64, np.float64):
        return TSU_F64
    raise ValueError(f"unsupported dtype {dt!r}")


class TsuError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func}: {_NAMES.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("ld", C.c_int64), ("dx", C.c_double), ("dy", C.c_double)]


class Sing(C.Structure):
    _fields_ = [("kind", C.c_int32), ("power", C.c_int32), ("amp", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double)]


class Depth(C.Structure):
    _fields_ = [("background", C.c_double), ("eps", C.c_double), ("mollifier", C.c_int32), ("nsing", C.c_int32),
                ("sing", C.POINTER(Sing))]


class Medium(C.Structure):
    _fields_ = [("hx", C.c_void_p), ("hy", C.c_void_p), ("hx_max", C.c_double), ("hy_max", C.c_double),
                ("hx_min", C.c_double), ("hy_min", C.c_double)]


def medium(hx, hy, ext) -> Medium:
    """The tsu_medium of face arrays hx, hy with the extrema ``ext`` = [min hx, max hx, min hy,
    max hy] that tsu_make_depth returns."""
    return Medium(_ptr(hx), _ptr(hy), float(ext[1]), float(ext[3]), float(ext[0]), float(ext[2]))


class State(C.Structure):
    _fields_ = [("buf", C.c_void_p * 4), ("nbuf", C.c_int32), ("form", C.c_int32), ("cur", C.c_int32),
                ("aux", C.c_int32), ("step", C.c_int64)]


class StepOpts(C.Structure):
    _fields_ = [("energy", C.c_void_p), ("nrec", C.c_int32), ("rec_idx", C.c_void_p), ("traces", C.c_void_p),
                ("ckpt", C.c_void_p), ("ckpt_every", C.c_int64), ("ckpt_slots", C.c_int64), ("kernel", C.c_int32),
                ("rows", C.c_int32), ("tdepth", C.c_int32), ("reserved", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("grid", Grid), ("tau", C.c_double), ("medium", Medium), ("state", C.POINTER(State)),
                ("nsteps", C.c_int64)]


class BatchOpts(C.Structure):
    _fields_ = [("tdepth", C.c_int32), ("rows", C.c_int32), ("kernel", C.c_int32), ("graph", C.c_int32),
                ("order", C.c_int32), ("rows_per_problem", C.POINTER(C.c_int32))]


def _batch_opts(tdepth=0, rows=0, kernel=0, graph=False, order=0, rows_per_problem=None) -> BatchOpts:
    o = BatchOpts(int(tdepth), int(rows), int(kernel), int(bool(graph)), int(order))
    if rows_per_problem is not None:
        arr = (C.c_int32 * len(rows_per_problem))(*[int(r) for r in rows_per_problem])
        o.rows_per_problem = C.cast(arr, C.POINTER(C.c_int32))
        o._keep = arr
    return o


_lib = None


def load():
    """Load libtsu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtsu.so not built ({LIB_PATH}); run paper_2005_11931_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "tsu_version": ([], C.c_int),
        "tsu_last_error": ([], C.c_char_p),
        "tsu_make_depth": ([C.POINTER(Grid), C.POINTER(Depth), C.c_int, vp, vp, vp, C.POINTER(C.c_double), vp], C.c_int),
        "tsu_tau_for": ([C.POINTER(Grid), dbl, dbl, dbl], dbl),
        "tsu_tau_courant": ([C.POINTER(Grid), C.POINTER(Medium), dbl], dbl),
        "tsu_depth_eps_derivative": ([C.POINTER(Grid), C.POINTER(Depth), C.c_int, vp, vp, vp], C.c_int),
        "tsu_reduce_workspace": ([], C.c_size_t),
        "tsu_depth_eps_gradient": ([C.POINTER(Grid), C.POINTER(Depth), vp, vp, vp, vp, C.c_size_t, vp], C.c_int),
        "tsu_diff_norms": ([C.POINTER(Grid), C.c_int, vp, vp, vp, vp, C.c_size_t, vp], C.c_int),
        "tsu_init": ([C.POINTER(Grid), C.c_int, dbl, C.POINTER(Medium), vp, vp, C.POINTER(State), vp], C.c_int),
        "tsu_step_workspace": ([C.POINTER(Grid), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "tsu_step_n": ([C.POINTER(Grid), C.c_int, dbl, C.POINTER(Medium), C.POINTER(State), i64,
                        C.POINTER(StepOpts), vp, C.c_size_t, vp], C.c_int),
        "tsu_sync_status": ([vp, C.c_size_t, vp], C.c_int),
        "tsu_ckpt_slots": ([i64, i64], i64),
        "tsu_aux_streams": ([], C.c_int),
        "tsu_step_n_noalloc": ([C.POINTER(Grid), C.c_int, dbl, C.POINTER(Medium), C.POINTER(State), i64, vp, vp],
                               C.c_int),
        "tsu_noalloc_last_error": ([], C.c_char_p),
        "tsu_batch_workspace": ([i32, C.POINTER(Problem), C.POINTER(BatchOpts), C.POINTER(C.c_size_t)], C.c_int),
        "tsu_batch_run": ([i32, C.POINTER(Problem), C.POINTER(BatchOpts), vp, C.c_size_t, vp], C.c_int),
        "tsu_adjoint_workspace": ([C.POINTER(Grid), C.c_int, C.c_int, i64, i64, i32, C.POINTER(C.c_size_t)],
                                  C.c_int),
        "tsu_adjoint": ([C.POINTER(Grid), C.c_int, C.c_int, dbl, C.POINTER(Medium), i64, i64, vp, vp, i32, vp, vp,
                         vp, vp, vp, vp, vp, C.c_size_t, vp], C.c_int),
        "tsu_observe": ([C.POINTER(Grid), C.c_int, dbl, C.POINTER(Medium), C.POINTER(State), vp, i32, vp, vp, vp,
                         C.c_size_t, vp], C.c_int),
        "tsu_implicit_sizes": ([C.POINTER(Grid), C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)], C.c_int),
        "tsu_implicit_factor": ([C.POINTER(Grid), C.c_int, dbl, dbl, C.POINTER(Medium), vp, C.c_size_t, vp], C.c_int),
        "tsu_implicit_init": ([C.POINTER(Grid), C.c_int, dbl, dbl, C.POINTER(Medium), vp, vp, vp, C.POINTER(State),
                               vp, C.c_size_t, vp], C.c_int),
        "tsu_implicit_step_n": ([C.POINTER(Grid), C.c_int, dbl, dbl, C.POINTER(Medium), vp, C.POINTER(State), i64,
                                 vp, C.c_size_t, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    """Entry points declared in include/tsu.h (parsed from the header text)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "tsu.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|double|size_t|const char\*)\s+(tsu_\w+)\s*\(", text, re.M)))


def _check(rc: int, func: str):
    if rc != TSU_OK:
        raise TsuError(rc, func, load().tsu_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    return int(t)


# The C ABI takes raw device addresses and cannot see how large a buffer is, so every tensor that
# crosses it is checked here first (device, element type, contiguity, size).  Plain integers are
# passed through as device addresses: their extent is the caller's responsibility.
def _checked(t, name: str, dtype, need: int):
    if t is None or not isinstance(t, torch.Tensor):
        return _ptr(t)
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype} (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < need:
        raise ValueError(f"{name} holds {t.numel()} elements; {need} are needed")
    return t.data_ptr()


def _field(t, g: "Grid", code: int, name: str):
    """A [ny][ld] device field of element type ``code``."""
    return _checked(t, name, DTYPES[code], int(g.ny) * int(g.ld))


def _vec(t, n: int, dtype, name: str):
    """A device vector of at least ``n`` elements of ``dtype`` (None: any element type)."""
    return _checked(t, name, dtype, int(n))


def _bytes(t, n: int, name: str):
    """A device byte buffer of at least ``n`` bytes (any element type)."""
    if isinstance(t, torch.Tensor):
        _checked(t, name, None, 0)
        if t.numel() * t.element_size() < n:
            raise ValueError(f"{name} holds {t.numel() * t.element_size()} bytes; {n} are needed")
    return _ptr(t)


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def grid(n: int, ny: int | None = None, ld: int | None = None) -> Grid:
    """Unit box with n x ny nodes (boundary included), rows padded to a multiple of 32."""
    ny = ny or n
    ld = ld or (n + 31) // 32 * 32
    return Grid(n, ny, ld, 1.0 / (n - 1), 1.0 / (ny - 1))


def depth_struct(depth: dict):
    sings = depth.get("sings", [])
    arr = (Sing * max(1, len(sings)))(*[Sing(*s) for s in sings])
    d = Depth(float(depth["background"]), float(depth["eps"]), int(depth.get("mollifier", TSU_GAUSS)), len(sings),
              C.cast(arr, C.POINTER(Sing)))
    d._keep = arr
    return d


def empty_field(g: Grid, dtype, device="cuda") -> torch.Tensor:
    return torch.zeros((g.ny, g.ld), dtype=DTYPES[dtype_code(dtype)], device=device)


# ---------------------------------------------------------------------------------------------
# C entry points
# ---------------------------------------------------------------------------------------------
def tsu_make_depth(g: Grid, depth: dict, dtype, hx: torch.Tensor, hy: torch.Tensor, ext_dev: torch.Tensor,
                   sync: bool = True, stream=None):
    """Face coefficients of the regularised depth; returns [min hx, max hx, min hy, max hy] when sync."""
    d = depth_struct(depth)
    code = dtype_code(dtype)
    ext = (C.c_double * 4)() if sync else None
    rc = load().tsu_make_depth(C.byref(g), C.byref(d), code, _field(hx, g, code, "hx"), _field(hy, g, code, "hy"),
                               _vec(ext_dev, 4, torch.float64, "ext_dev"), ext, _stream(stream))
    _check(rc, "tsu_make_depth")
    return np.array(list(ext)) if sync else None


def tsu_depth_eps_derivative(g: Grid, depth: dict, dtype, dhx: torch.Tensor, dhy: torch.Tensor, stream=None):
    """d h_eps / d eps at the faces, same layout as tsu_make_depth's hx, hy."""
    d = depth_struct(depth)
    code = dtype_code(dtype)
    _check(load().tsu_depth_eps_derivative(C.byref(g), C.byref(d), code, _field(dhx, g, code, "dhx"),
                                           _field(dhy, g, code, "dhy"), _stream(stream)), "tsu_depth_eps_derivative")


def tsu_reduce_workspace() -> int:
    return int(load().tsu_reduce_workspace())


def _ws_bytes(ws, ws_bytes):
    if ws_bytes is not None:
        return int(ws_bytes)
    return int(ws.numel() * ws.element_size()) if isinstance(ws, torch.Tensor) else 0


def tsu_depth_eps_gradient(g: Grid, depth: dict, g_hx: torch.Tensor, g_hy: torch.Tensor, out: torch.Tensor,
                           ws: torch.Tensor, stream=None, ws_bytes=None):
    """out[0] = dJ/deps = sum g_hx dhx/deps + g_hy dhy/deps (device double)."""
    d = depth_struct(depth)
    wsb = _ws_bytes(ws, ws_bytes)
    _check(load().tsu_depth_eps_gradient(C.byref(g), C.byref(d), _field(g_hx, g, TSU_F64, "g_hx"),
                                         _field(g_hy, g, TSU_F64, "g_hy"), _vec(out, 1, torch.float64, "out"),
                                         _bytes(ws, wsb, "ws"), wsb, _stream(stream)),
           "tsu_depth_eps_gradient")


def tsu_diff_norms(g: Grid, dtype, a: torch.Tensor, b: torch.Tensor, out: torch.Tensor, ws: torch.Tensor,
                   stream=None, ws_bytes=None):
    """out[0] = sum (a - b)^2, out[1] = sum b^2 over nodes i < nx (device double[2])."""
    code = dtype_code(dtype)
    wsb = _ws_bytes(ws, ws_bytes)
    _check(load().tsu_diff_norms(C.byref(g), code, _field(a, g, code, "a"), _field(b, g, code, "b"),
                                 _vec(out, 2, torch.float64, "out"), _bytes(ws, wsb, "ws"), wsb, _stream(stream)),
           "tsu_diff_norms")


def tsu_tau_for(g: Grid, hx_max: float, hy_max: float, cfl: float) -> float:
    return float(load().tsu_tau_for(C.byref(g), hx_max, hy_max, cfl))


def tsu_tau_courant(g: Grid, medium: Medium, courant: float) -> float:
    """tau = courant min(dx, dy) / sqrt(max face depth), the workloads' time step (0 on bad input)."""
    return float(load().tsu_tau_courant(C.byref(g), C.byref(medium), float(courant)))


def tsu_init(g: Grid, dtype, tau: float, medium: Medium, u0, u1, state: State, stream=None):
    code = dtype_code(dtype)
    rc = load().tsu_init(C.byref(g), code, tau, C.byref(medium), _field(u0, g, code, "u0"),
                         _field(u1, g, code, "u1"), C.byref(state), _stream(stream))
    _check(rc, "tsu_init")


def tsu_step_workspace(g: Grid, dtype) -> int:
    n = C.c_size_t(0)
    _check(load().tsu_step_workspace(C.byref(g), dtype_code(dtype), C.byref(n)), "tsu_step_workspace")
    return int(n.value)


def tsu_step_n(g: Grid, dtype, tau: float, medium: Medium, state: State, nsteps: int, opts: StepOpts | None = None,
               ws=None, ws_bytes: int = 0, stream=None):
    rc = load().tsu_step_n(C.byref(g), dtype_code(dtype), tau, C.byref(medium), C.byref(state), int(nsteps),
                           C.byref(opts) if opts is not None else None, _ptr(ws), int(ws_bytes), _stream(stream))
    _check(rc, "tsu_step_n")


def tsu_sync_status(ws, ws_bytes: int, stream=None):
    """Synchronise and raise TsuError if a kernel recorded an expired bounded wait."""
    _check(load().tsu_sync_status(_ptr(ws), int(ws_bytes), _stream(stream)), "tsu_sync_status")


def _problems(sims, nsteps):
    arr = (Problem * len(sims))()
    for k, (sim, n) in enumerate(zip(sims, nsteps)):
        arr[k].grid = sim.g
        arr[k].tau = sim.tau
        arr[k].medium = sim.medium
        arr[k].state = C.pointer(sim.state)
        arr[k].nsteps = int(n)
    return arr


def tsu_batch_workspace(sims, nsteps, tdepth: int = 0, rows: int = 0, kernel: int = 0, order: int = 0,
                        rows_per_problem=None) -> int:
    arr = _problems(sims, nsteps)
    o = _batch_opts(tdepth, rows, kernel, False, order, rows_per_problem)
    n = C.c_size_t(0)
    _check(load().tsu_batch_workspace(len(sims), arr, C.byref(o), C.byref(n)), "tsu_batch_workspace")
    return int(n.value)


def tsu_batch_run(sims, nsteps, ws, ws_bytes: int, tdepth: int = 0, rows: int = 0, kernel: int = 0,
                  graph: bool = False, order: int = 0, rows_per_problem=None, stream=None):
    """Advance every Simulation in ``sims`` by its entry of ``nsteps`` in batched launches (captured
    into one CUDA graph when ``graph``; that needs a non-default stream).  ``order`` and
    ``rows_per_problem`` pack the tiles (tsu_batch_opts)."""
    arr = _problems(sims, nsteps)
    o = _batch_opts(tdepth, rows, kernel, graph, order, rows_per_problem)
    rc = load().tsu_batch_run(len(sims), arr, C.byref(o), _bytes(ws, ws_bytes, "ws"), int(ws_bytes),
                              _stream(stream))
    _check(rc, "tsu_batch_run")


def batch_run(sims, nsteps, tune: bool = False, cache=None, stream=None, **opts):
    """tsu_batch_run with a workspace of its own.  ``tune``: the configuration the autotuner picks
    for these problems (timed once on scratch copies, then cached); otherwise ``opts`` (tdepth,
    rows, kernel, graph, order, rows_per_problem) or the library's defaults.  Returns the options
    used."""
    if tune:
        from . import autotune
        opts = autotune.tune_batch(sims, cache=cache).batch_opts(sims)
    dev = sims[0].hx.device
    wsb = tsu_batch_workspace(sims, nsteps, **{k: v for k, v in opts.items() if k != "graph"})
    ws = torch.zeros(wsb, dtype=torch.uint8, device=dev)
    tsu_batch_run(sims, nsteps, ws, wsb, stream=stream, **opts)
    return opts


def tsu_step_n_noalloc(g: Grid, dtype, tau: float, medium: Medium, state: State, nsteps: int, energy=None,
                       stream=None):
    """tsu_step_n (one step per pass, optional energy) without a caller workspace."""
    lib = load()
    rc = lib.tsu_step_n_noalloc(C.byref(g), dtype_code(dtype), tau, C.byref(medium), C.byref(state), int(nsteps),
                                _vec(energy, nsteps, torch.float64, "energy"), _stream(stream))
    if rc != TSU_OK:
        raise TsuError(rc, "tsu_step_n_noalloc", lib.tsu_noalloc_last_error().decode())


def tsu_aux_streams() -> int:
    """Auxiliary recompute streams the library holds (one per device and host thread that ran an adjoint)."""
    return int(load().tsu_aux_streams())


def tsu_ckpt_slots(nsteps: int, ckpt_every: int) -> int:
    return int(load().tsu_ckpt_slots(int(nsteps), int(ckpt_every)))


def tsu_adjoint_workspace(g: Grid, dtype, form: int, nsteps: int, ckpt_every: int, nrec: int = 0) -> int:
    n = C.c_size_t(0)
    _check(load().tsu_adjoint_workspace(C.byref(g), dtype_code(dtype), int(form), int(nsteps), int(ckpt_every),
                                        int(nrec), C.byref(n)), "tsu_adjoint_workspace")
    return int(n.value)


def tsu_adjoint(g: Grid, dtype, form: int, tau: float, medium: Medium, nsteps: int, ckpt_every: int, ckpt, u0,
                rec_idx, dtraces, g_hx, g_hy, g_u0, g_u1, ws, ws_bytes: int, stream=None):
    nrec = 0 if rec_idx is None else int(rec_idx.numel())
    code = dtype_code(dtype)
    fields = int(g.ny) * int(g.ld)
    slots = tsu_ckpt_slots(nsteps, ckpt_every)
    rc = load().tsu_adjoint(C.byref(g), code, int(form), tau, C.byref(medium), int(nsteps), int(ckpt_every),
                            _vec(ckpt, 2 * slots * fields, DTYPES[code], "ckpt"), _field(u0, g, code, "u0"), nrec,
                            _vec(rec_idx, nrec, torch.int64, "rec_idx"),
                            _vec(dtraces, int(nsteps) * nrec, DTYPES[code], "dtraces"),
                            _field(g_hx, g, TSU_F64, "g_hx"), _field(g_hy, g, TSU_F64, "g_hy"),
                            _field(g_u0, g, code, "g_u0"), _field(g_u1, g, code, "g_u1"), _bytes(ws, ws_bytes, "ws"),
                            int(ws_bytes), _stream(stream))
    _check(rc, "tsu_adjoint")


def tsu_observe(g: Grid, dtype, tau: float, medium: Medium, state: State, energy_dev=None, rec_idx=None,
                trace=None, ws=None, ws_bytes: int = 0, stream=None):
    nrec = 0 if rec_idx is None else int(rec_idx.numel())
    code = dtype_code(dtype)
    rc = load().tsu_observe(C.byref(g), code, tau, C.byref(medium), C.byref(state),
                            _vec(energy_dev, 1, torch.float64, "energy"), nrec,
                            _vec(rec_idx, nrec, torch.int64, "rec_idx"), _vec(trace, nrec, DTYPES[code], "trace"),
                            _bytes(ws, ws_bytes, "ws"), int(ws_bytes), _stream(stream))
    _check(rc, "tsu_observe")


# ---------------------------------------------------------------------------------------------
# Convenience: one forward problem with torch-owned buffers
# ---------------------------------------------------------------------------------------------
def tsu_implicit_sizes(g: Grid, dtype) -> tuple[int, int]:
    fb, wb = C.c_size_t(0), C.c_size_t(0)
    _check(load().tsu_implicit_sizes(C.byref(g), dtype_code(dtype), C.byref(fb), C.byref(wb)), "tsu_implicit_sizes")
    return int(fb.value), int(wb.value)


def tsu_implicit_factor(g: Grid, dtype, tau: float, sigma: float, medium: Medium, factor, factor_bytes: int,
                        stream=None):
    _check(load().tsu_implicit_factor(C.byref(g), dtype_code(dtype), float(tau), float(sigma), C.byref(medium),
                                      _ptr(factor), int(factor_bytes), _stream(stream)), "tsu_implicit_factor")


def tsu_implicit_init(g: Grid, dtype, tau: float, sigma: float, medium: Medium, factor, u0, u1, state: State, ws,
                      ws_bytes: int, stream=None):
    code = dtype_code(dtype)
    _check(load().tsu_implicit_init(C.byref(g), code, float(tau), float(sigma), C.byref(medium),
                                    _ptr(factor), _field(u0, g, code, "u0"), _field(u1, g, code, "u1"),
                                    C.byref(state), _bytes(ws, ws_bytes, "ws"), int(ws_bytes), _stream(stream)),
           "tsu_implicit_init")


def tsu_implicit_step_n(g: Grid, dtype, tau: float, sigma: float, medium: Medium, factor, state: State, nsteps: int,
                        ws, ws_bytes: int, stream=None):
    _check(load().tsu_implicit_step_n(C.byref(g), dtype_code(dtype), float(tau), float(sigma), C.byref(medium),
                                      _ptr(factor), C.byref(state), int(nsteps), _ptr(ws), int(ws_bytes),
                                      _stream(stream)), "tsu_implicit_step_n")


class ImplicitSimulation:
    """Buffers and calls of one problem stepped by the implicit comparator (marshalling only):
    the depth, the line systems' factor, the workspace and the state (u, v)."""

    def __init__(self, g, dtype, hx, hy, ext, tau, sigma, medium, factor, ws, bufs, state):
        self.g, self.dtype, self.hx, self.hy, self.ext = g, dtype, hx, hy, ext
        self.tau, self.sigma, self.medium = tau, sigma, medium
        self.factor, self.ws, self.bufs, self.state = factor, ws, bufs, state

    @classmethod
    def create(cls, n: int, depth: dict, dtype="f64", tau=None, cfl: float = 0.4, sigma: float = 0.25, ny=None,
               ld=None, stream=None, device="cuda"):
        g = grid(n, ny, ld)
        code = dtype_code(dtype)
        hx = empty_field(g, code, device)
        hy = empty_field(g, code, device)
        ext_dev = torch.zeros(4, dtype=torch.float64, device=device)
        ext = tsu_make_depth(g, depth, code, hx, hy, ext_dev, sync=True, stream=stream)
        med = medium(hx, hy, ext)
        if tau is None:
            tau = tsu_tau_courant(g, med, cfl)
        fb, wb = tsu_implicit_sizes(g, code)
        factor = torch.empty(fb, dtype=torch.uint8, device=device)
        ws = torch.zeros(wb, dtype=torch.uint8, device=device)  # the status word starts at 0
        tsu_implicit_factor(g, code, tau, sigma, med, factor, fb, stream)
        bufs = [empty_field(g, code, device) for _ in range(2)]
        st = State()
        for k, b in enumerate(bufs):
            st.buf[k] = b.data_ptr()
        st.nbuf = 2
        st.form = TSU_FORM_INCREMENT
        return cls(g, code, hx, hy, ext, float(tau), float(sigma), med, factor, ws, bufs, st)

    def init(self, u0: torch.Tensor, u1: torch.Tensor | None = None, stream=None):
        tsu_implicit_init(self.g, self.dtype, self.tau, self.sigma, self.medium, self.factor, u0, u1, self.state,
                          self.ws, self.ws.numel(), stream)

    def step(self, nsteps: int, stream=None):
        tsu_implicit_step_n(self.g, self.dtype, self.tau, self.sigma, self.medium, self.factor, self.state, nsteps,
                            self.ws, self.ws.numel(), stream)

    @property
    def u(self) -> torch.Tensor:
        return self.bufs[self.state.cur]

    @property
    def v(self) -> torch.Tensor:
        return self.bufs[self.state.aux]


@dataclass
class Simulation:
    """Buffers and calls of one forward problem (marshalling only)."""
    g: Grid
    dtype: int
    form: int
    hx: torch.Tensor
    hy: torch.Tensor
    ext: np.ndarray
    tau: float
    medium: Medium
    bufs: list
    state: State
    ws: torch.Tensor

    @classmethod
    def create(cls, n: int, depth: dict, dtype="f32", form=None, cfl: float = 0.4, tau=None,
               ny=None, ld=None, stream=None, device="cuda", nbuf=None):
        g = grid(n, ny, ld)
        code = dtype_code(dtype)
        if form is None:  # FP32 fields keep their accuracy over long runs in the increment form
            form = TSU_FORM_INCREMENT if code == TSU_F32 else TSU_FORM_STANDARD
        hx = empty_field(g, code, device)
        hy = empty_field(g, code, device)
        ext_dev = torch.zeros(4, dtype=torch.float64, device=device)
        ext = tsu_make_depth(g, depth, code, hx, hy, ext_dev, sync=True, stream=stream)
        med = medium(hx, hy, ext)
        if tau is None:  # the workloads' rule (tsu_tau_courant): cfl min(dx, dy) / sqrt(max face depth)
            tau = tsu_tau_courant(g, med, cfl)
        nb = 4 if nbuf is None else nbuf
        bufs = [empty_field(g, code, device) for _ in range(nb)]
        st = State()
        for k, b in enumerate(bufs):
            st.buf[k] = b.data_ptr()
        st.nbuf = nb
        st.form = form
        ws_bytes = tsu_step_workspace(g, code)
        ws = torch.zeros(ws_bytes, dtype=torch.uint8, device=device)
        return cls(g, code, form, hx, hy, ext, float(tau), med, bufs, st, ws)

    def init(self, u0: torch.Tensor, u1: torch.Tensor | None = None, stream=None):
        tsu_init(self.g, self.dtype, self.tau, self.medium, u0, u1, self.state, stream)

    def step(self, nsteps: int, energy: torch.Tensor | None = None, rec_idx: torch.Tensor | None = None,
             traces: torch.Tensor | None = None, ckpt: torch.Tensor | None = None, ckpt_every: int = 0,
             kernel: int = 0, rows: int = 0, tdepth: int = 0, debug: int = 0, stream=None):
        o = StepOpts()
        nrec = 0 if rec_idx is None else int(rec_idx.numel())
        fdt = DTYPES[self.dtype]
        o.energy = _vec(energy, nsteps, torch.float64, "energy")
        o.nrec = nrec
        o.rec_idx = _vec(rec_idx, nrec, torch.int64, "rec_idx")
        o.traces = _vec(traces, int(nsteps) * nrec, fdt, "traces")
        if ckpt is not None and tuple(ckpt.shape[1:]) != (2, self.g.ny, self.g.ld):
            raise ValueError(f"ckpt must be [slots][2][ny][ld] (got {tuple(ckpt.shape)})")
        o.ckpt = _vec(ckpt, 0, fdt, "ckpt")
        o.ckpt_every = int(ckpt_every)
        o.ckpt_slots = 0 if ckpt is None else int(ckpt.shape[0])
        o.kernel, o.rows, o.tdepth, o.reserved = int(kernel), int(rows), int(tdepth), int(debug)
        tsu_step_n(self.g, self.dtype, self.tau, self.medium, self.state, nsteps, o, self.ws, self.ws.numel(), stream)

    def observe(self, energy: torch.Tensor | None = None, rec_idx=None, trace=None, stream=None):
        tsu_observe(self.g, self.dtype, self.tau, self.medium, self.state, energy, rec_idx, trace, self.ws,
                    self.ws.numel(), stream)

    def clone(self) -> "Simulation":
        """A copy with its own state buffers and workspace (same medium, tau and roles)."""
        bufs = [b.clone() for b in self.bufs]
        st = State()
        for k, b in enumerate(bufs):
            st.buf[k] = b.data_ptr()
        st.nbuf, st.form, st.cur, st.aux, st.step = (self.state.nbuf, self.state.form, self.state.cur,
                                                     self.state.aux, self.state.step)
        return Simulation(self.g, self.dtype, self.form, self.hx, self.hy, self.ext, self.tau, self.medium, bufs, st,
                          torch.zeros_like(self.ws))

    @property
    def u_prev(self) -> torch.Tensor | None:
        """u^{n-1} (standard form only)."""
        return self.bufs[self.state.aux] if self.form == TSU_FORM_STANDARD else None

    @property
    def v(self) -> torch.Tensor | None:
        """v^n = u^n - u^{n-1} (increment form only)."""
        return self.bufs[self.state.aux] if self.form == TSU_FORM_INCREMENT else None

    @property
    def u(self) -> torch.Tensor:
        """u^n (current level)."""
        return self.bufs[self.state.cur]
