"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/tsu.h
declares.  No GPU: no compute call is made here."""
import ctypes as C
import re

from paper_2005_11931_gb300 import build, tsu


def test_library_builds_and_exports_declared_symbols():
    path = build.build()
    lib = C.CDLL(path)
    names = tsu.declared_symbols()
    assert "tsu_step_n" in names and "tsu_make_depth" in names and "tsu_init" in names
    for n in names:
        assert hasattr(lib, n), n


def test_host_only_entry_points():
    lib = tsu.load()
    assert lib.tsu_version() >= 100
    g = tsu.grid(201)
    # leapfrog bound tau^2 (hx/dx^2 + hy/dy^2) <= 1
    t = tsu.tsu_tau_for(g, 2.0, 2.0, 1.0)
    assert abs(t * t * (2.0 / g.dx ** 2 + 2.0 / g.dy ** 2) - 1.0) < 1e-14
    assert tsu.tsu_tau_for(g, 2.0, 2.0, 1.5) == 0.0
    assert tsu.tsu_step_workspace(g, tsu.TSU_F32) > 256


def test_binding_structs_match_header_layout():
    """Field order and sizes of the ctypes mirrors follow the header text."""
    hdr = open(tsu.declared_symbols.__code__.co_filename.replace("paper_2005_11931_gb300/tsu.py",
                                                                 "include/tsu.h")).read()
    assert C.sizeof(tsu.Grid) == 32 and C.sizeof(tsu.Sing) == 32
    assert C.sizeof(tsu.State) == 4 * 8 + 4 * 4 + 8
    for struct, cname in ((tsu.StepOpts, "tsu_step_opts"), (tsu.State, "tsu_state"), (tsu.Medium, "tsu_medium")):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)(?:\[\d+\])?\s*[;,]", body)
        assert [f[0] for f in struct._fields_] == fields, (cname, fields)


def test_implicit_sizes_and_argument_checks_on_the_host():
    """The implicit comparator's size query, and the argument checks that refuse a call before any
    device work (no GPU: the pointers are never dereferenced, the stream is the null handle)."""
    import pytest

    g = tsu.grid(131, 77)  # ld 160, transposed rows of roundup(77, 32) = 96
    fb, wb = tsu.tsu_implicit_sizes(g, tsu.TSU_F32)
    ldT = 96
    assert fb == 4 * (77 * 160 + 2 * 131 * ldT)
    assert wb == 4 * (131 * ldT + max(77 * 160, 131 * ldT))
    fb64, wb64 = tsu.tsu_implicit_sizes(g, tsu.TSU_F64)
    assert (fb64, wb64) == (2 * fb, 2 * wb)
    fake = 1 << 20  # 16-byte aligned, never touched
    med = tsu.Medium(fake, fake, 2.0, 2.0)
    with pytest.raises(tsu.TsuError) as e:  # weight below 0
        tsu.tsu_implicit_factor(g, tsu.TSU_F32, 0.01, -0.1, med, fake, fb, stream=0)
    assert e.value.code == tsu.TSU_EINVAL
    with pytest.raises(tsu.TsuError) as e:  # weight below 1/4 beyond its Courant bound
        tsu.tsu_implicit_factor(g, tsu.TSU_F32, 1.0, 0.0, med, fake, fb, stream=0)
    assert e.value.code == tsu.TSU_ECFL
    with pytest.raises(tsu.TsuError) as e:  # factor buffer too small
        tsu.tsu_implicit_factor(g, tsu.TSU_F32, 1.0, 0.25, med, fake, fb - 4, stream=0)
    assert e.value.code == tsu.TSU_ENOMEM
    with pytest.raises(tsu.TsuError) as e:  # misaligned factor
        tsu.tsu_implicit_factor(g, tsu.TSU_F32, 1.0, 0.25, med, fake + 4, fb, stream=0)
    assert e.value.code == tsu.TSU_EINVAL
    st = tsu.State()
    st.buf[0], st.buf[1], st.nbuf, st.form = fake, fake + 4096, 2, tsu.TSU_FORM_STANDARD
    with pytest.raises(tsu.TsuError) as e:  # the implicit scheme runs in the increment form
        tsu.tsu_implicit_init(g, tsu.TSU_F32, 1.0, 0.25, med, fake, fake, None, st, fake, wb, stream=0)
    assert e.value.code == tsu.TSU_EINVAL
    st.form = tsu.TSU_FORM_INCREMENT
    with pytest.raises(tsu.TsuError) as e:  # workspace too small
        tsu.tsu_implicit_init(g, tsu.TSU_F32, 1.0, 0.25, med, fake, fake, None, st, fake, wb - 16, stream=0)
    assert e.value.code == tsu.TSU_ENOMEM
    st.cur, st.aux = 0, 0
    with pytest.raises(tsu.TsuError) as e:  # roles must differ
        tsu.tsu_implicit_step_n(g, tsu.TSU_F32, 1.0, 0.25, med, fake, st, 5, fake, wb, stream=0)
    assert e.value.code == tsu.TSU_EINVAL
    st.cur, st.aux = 0, 1
    tsu.tsu_implicit_step_n(g, tsu.TSU_F32, 1.0, 0.25, med, fake, st, 0, fake, wb, stream=0)  # nothing to do
    assert st.step == 0
