"""Argument checks of the C ABI that refuse a call before any device work.

These functions hand the library addresses that point nowhere (plain integers, never
dereferenced) and grids far larger than any buffer.  They must therefore never run where a GPU is
visible: if a check regressed, or moved behind a launch, a kernel would read and write through
those addresses on a shared device.  tests/test_abi.py runs each of them in a child process whose
CUDA_VISIBLE_DEVICES is empty, where a regression surfaces as TSU_ECUDA ("no device") instead.
"""
from __future__ import annotations

import math
import os

from paper_2005_11931_gb300 import tsu

FAKE = 1 << 20  # 16-byte aligned, never touched


def _expect(code, fn, *args, **kw):
    try:
        fn(*args, **kw)
    except tsu.TsuError as e:
        assert e.code == code, (fn.__name__, e)
        return str(e)
    raise AssertionError(f"{fn.__name__} accepted arguments it must refuse")


def _state(nbuf=2, form=tsu.TSU_FORM_STANDARD, cur=1, aux=0):
    st = tsu.State()
    for k in range(nbuf):
        st.buf[k] = FAKE + 4096 * k
    st.nbuf, st.form, st.cur, st.aux = nbuf, form, cur, aux
    return st


def no_device_visible():
    assert os.environ.get("CUDA_VISIBLE_DEVICES") == "", "run these checks where no GPU is visible"


def noalloc_refuses_beyond_its_fixed_scratch():
    """FP64 on 32800 x 32800 needs ceil(32800/256) * ceil(32798/32) = 129 * 1025 > 65536 energy
    partials; refused with TSU_ENOMEM, and the same grid without an energy output passes the
    checks (nsteps = 0: nothing to enqueue)."""
    no_device_visible()
    g = tsu.Grid(32800, 32800, 32800, 1 / 32799, 1 / 32799)
    med = tsu.Medium(FAKE, FAKE, 1.0, 1.0, 1.0, 1.0)
    msg = _expect(tsu.TSU_ENOMEM, tsu.tsu_step_n_noalloc, g, "f64", 1e-6, med, _state(), 1, energy=FAKE, stream=0)
    assert "too large" in msg
    tsu.tsu_step_n_noalloc(g, "f64", 1e-6, med, _state(), 0, energy=None, stream=0)


def both_stepping_entry_points_refuse_the_same_inputs():
    """tsu_step_n and tsu_step_n_noalloc share their argument checks: a non-finite tau, a medium
    whose extrema break positivity, a step outside the leapfrog bound and bad state roles are
    refused by both with the same status."""
    no_device_visible()
    g = tsu.grid(257)
    ok = tsu.Medium(FAKE, FAKE, 1.0, 1.0, 0.5, 0.5)
    tau = 0.4 * g.dx
    cases = [
        (tsu.TSU_EINVAL, tsu.grid(257), math.inf, ok, _state()),      # tau = inf
        (tsu.TSU_EINVAL, tsu.grid(257), math.nan, ok, _state()),      # tau = nan
        (tsu.TSU_EINVAL, tsu.grid(257), -tau, ok, _state()),          # tau < 0
        (tsu.TSU_ENONPOS, tsu.grid(257), tau, tsu.Medium(FAKE, FAKE, 1.0, 1.0, 0.0, 0.5), _state()),
        (tsu.TSU_ENONPOS, tsu.grid(257), tau, tsu.Medium(FAKE, FAKE, 1.0, 1.0, -0.1, 0.5), _state()),
        (tsu.TSU_ENONPOS, tsu.grid(257), tau, tsu.Medium(FAKE, FAKE, 0.0, 0.0, 0.0, 0.0), _state()),
        (tsu.TSU_ENONPOS, tsu.grid(257), tau, tsu.Medium(FAKE, FAKE, 1.0, 1.0, 2.0, 0.5), _state()),  # min > max
        (tsu.TSU_EINVAL, tsu.grid(257), tau, tsu.Medium(FAKE, FAKE, math.inf, 1.0, 0.5, 0.5), _state()),
        (tsu.TSU_ECFL, tsu.grid(257), 2 * g.dx, ok, _state()),        # tau^2 (1/dx^2 + 1/dy^2) = 8 > 1
        (tsu.TSU_EINVAL, tsu.grid(257), tau, ok, _state(cur=0, aux=0)),
        (tsu.TSU_EINVAL, tsu.Grid(257, 257, 258, g.dx, g.dy), tau, ok, _state()),            # ld % 4 != 0
        (tsu.TSU_EINVAL, tsu.Grid(257, 2 ** 31 - 1, 1024, g.dx, g.dy), tau, ok, _state()),   # >= 2^40 elements
        (tsu.TSU_EINVAL, tsu.grid(257), tau, tsu.Medium(FAKE + 4, FAKE, 1.0, 1.0, 0.5, 0.5), _state()),
    ]
    for code, gg, t, med, st in cases:
        a = _expect(code, tsu.tsu_step_n, gg, "f32", t, med, st, 3, None, None, 0, stream=0)
        b = _expect(code, tsu.tsu_step_n_noalloc, gg, "f32", t, med, _state(st.nbuf, st.form, st.cur, st.aux), 3,
                    energy=None, stream=0)
        assert a.split(": ", 2)[-1] == b.split(": ", 2)[-1], (a, b)
    # a face family that is identically zero is the 1D reduction, not a positivity failure: with
    # nsteps = 0 nothing is enqueued and the call succeeds
    one_d = tsu.Medium(FAKE, FAKE, 1.0, 0.0, 1.0, 0.0)
    tsu.tsu_step_n(g, "f32", g.dx, one_d, _state(), 0, None, None, 0, stream=0)
    tsu.tsu_step_n_noalloc(g, "f32", g.dx, one_d, _state(), 0, energy=None, stream=0)


def init_refuses_a_nonpositive_medium():
    """tsu_init returns TSU_ENONPOS for a medium whose face minimum is <= 0 (Sec. 2 positivity),
    before anything is enqueued."""
    no_device_visible()
    g = tsu.grid(129)
    for med in (tsu.Medium(FAKE, FAKE, 1.0, 1.0, 0.0, 1.0), tsu.Medium(FAKE, FAKE, 1.0, 1.0, 1.0, -1e-3)):
        _expect(tsu.TSU_ENONPOS, tsu.tsu_init, g, "f32", 0.4 * g.dx, med, FAKE, None, _state(), stream=0)
    _expect(tsu.TSU_ENONPOS, tsu.tsu_observe, g, "f32", 0.4 * g.dx, tsu.Medium(FAKE, FAKE, 1.0, 1.0, 0.0, 1.0),
            _state(), FAKE, None, None, FAKE, 1 << 20, stream=0)


def workload_time_step_rule():
    """tsu_tau_courant: tau = courant min(dx, dy) / sqrt(max face depth)."""
    g = tsu.grid(201, 101)
    med = tsu.Medium(FAKE, FAKE, 29.2, 3.0, 1.0, 1.0)
    t = tsu.tsu_tau_courant(g, med, 0.4)
    assert t == 0.4 * min(g.dx, g.dy) / math.sqrt(29.2)
    assert tsu.tsu_tau_courant(g, tsu.Medium(FAKE, FAKE, 2.0, 7.0, 1.0, 1.0), 0.4) == 0.4 * g.dx / math.sqrt(7.0)
    assert tsu.tsu_tau_courant(g, med, 0.0) == 0.0
    assert tsu.tsu_tau_courant(g, med, math.inf) == 0.0
    assert tsu.tsu_tau_courant(g, tsu.Medium(FAKE, FAKE, 0.0, 0.0, 0.0, 0.0), 0.4) == 0.0
    # within the leapfrog bound for courant <= 1/sqrt(2)
    c = 1 / math.sqrt(2)
    tt = tsu.tsu_tau_courant(g, tsu.Medium(FAKE, FAKE, 5.0, 5.0, 1.0, 1.0), c)
    assert tt * tt * (5.0 / g.dx ** 2 + 5.0 / g.dy ** 2) <= 1.0 + 1e-15


def implicit_sizes_and_argument_checks():
    """The implicit comparator's size query, and the argument checks that refuse a call before any
    device work."""
    no_device_visible()
    g = tsu.grid(131, 77)  # ld 160, transposed rows of roundup(77, 32) = 96
    fb, wb = tsu.tsu_implicit_sizes(g, tsu.TSU_F32)
    ldT = 96
    assert fb == 4 * (77 * 160 + 2 * 131 * ldT)
    assert wb == 256 + 4 * (131 * ldT + max(77 * 160, 131 * ldT))  # a header with the status word first
    fb64, wb64 = tsu.tsu_implicit_sizes(g, tsu.TSU_F64)
    assert (fb64, wb64) == (2 * fb, 256 + 2 * (wb - 256))
    med = tsu.Medium(FAKE, FAKE, 2.0, 2.0, 1.0, 1.0)
    _expect(tsu.TSU_EINVAL, tsu.tsu_implicit_factor, g, tsu.TSU_F32, 0.01, -0.1, med, FAKE, fb, stream=0)
    _expect(tsu.TSU_ECFL, tsu.tsu_implicit_factor, g, tsu.TSU_F32, 1.0, 0.0, med, FAKE, fb, stream=0)
    _expect(tsu.TSU_ENOMEM, tsu.tsu_implicit_factor, g, tsu.TSU_F32, 1.0, 0.25, med, FAKE, fb - 4, stream=0)
    _expect(tsu.TSU_EINVAL, tsu.tsu_implicit_factor, g, tsu.TSU_F32, 1.0, 0.25, med, FAKE + 4, fb, stream=0)
    _expect(tsu.TSU_ENONPOS, tsu.tsu_implicit_factor, g, tsu.TSU_F32, 1.0, 0.25,
            tsu.Medium(FAKE, FAKE, 2.0, 2.0, 0.0, 1.0), FAKE, fb, stream=0)
    st = tsu.State()
    st.buf[0], st.buf[1], st.nbuf, st.form = FAKE, FAKE + 4096, 2, tsu.TSU_FORM_STANDARD
    # the implicit scheme runs in the increment form
    _expect(tsu.TSU_EINVAL, tsu.tsu_implicit_init, g, tsu.TSU_F32, 1.0, 0.25, med, FAKE, FAKE, None, st, FAKE, wb,
            stream=0)
    st.form = tsu.TSU_FORM_INCREMENT
    _expect(tsu.TSU_ENOMEM, tsu.tsu_implicit_init, g, tsu.TSU_F32, 1.0, 0.25, med, FAKE, FAKE, None, st, FAKE,
            wb - 16, stream=0)
    st.cur, st.aux = 0, 0  # roles must differ
    _expect(tsu.TSU_EINVAL, tsu.tsu_implicit_step_n, g, tsu.TSU_F32, 1.0, 0.25, med, FAKE, st, 5, FAKE, wb, stream=0)
    st.cur, st.aux = 0, 1
    tsu.tsu_implicit_step_n(g, tsu.TSU_F32, 1.0, 0.25, med, FAKE, st, 0, FAKE, wb, stream=0)  # nothing to do
    assert st.step == 0


def reductions_refuse_misaligned_fields():
    """tsu_diff_norms and tsu_depth_eps_gradient refuse a field that is not 16-byte aligned, and a
    workspace that is too small, before any device work."""
    no_device_visible()
    g = tsu.grid(100, 60)
    wsb = tsu.tsu_reduce_workspace()
    _expect(tsu.TSU_EINVAL, tsu.tsu_diff_norms, g, "f64", FAKE, FAKE + 8, FAKE, FAKE, stream=0, ws_bytes=wsb)
    _expect(tsu.TSU_ENOMEM, tsu.tsu_diff_norms, g, "f64", FAKE, FAKE, FAKE, FAKE, stream=0, ws_bytes=wsb - 8)
    depth = dict(background=1.0, eps=0.05, sings=[(0, 1, 1.0, 0.5, 0.5)])
    _expect(tsu.TSU_EINVAL, tsu.tsu_depth_eps_gradient, g, depth, FAKE + 8, FAKE, FAKE, FAKE, stream=0,
            ws_bytes=wsb)
    assert wsb > 256
