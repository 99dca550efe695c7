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
