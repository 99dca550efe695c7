"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/tsu.h
declares.  No GPU: no compute call is made here."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

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
    for struct, cname in ((tsu.StepOpts, "tsu_step_opts"), (tsu.State, "tsu_state"), (tsu.Medium, "tsu_medium"),
                          (tsu.BatchOpts, "tsu_batch_opts")):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)(?:\[\d+\])?\s*[;,]", body)
        assert [f[0] for f in struct._fields_] == fields, (cname, fields)


CHECKS = ["noalloc_refuses_beyond_its_fixed_scratch", "both_stepping_entry_points_refuse_the_same_inputs",
          "init_refuses_a_nonpositive_medium", "workload_time_step_rule", "implicit_sizes_and_argument_checks",
          "reductions_refuse_misaligned_fields"]


def test_argument_checks_without_a_device():
    """Refusals that happen before any device work, checked with addresses that point nowhere in a
    child process where no GPU is visible (a regression then fails with 'no device' and never
    touches a GPU).  Every function of tests/host_checks.py runs; each reports on its own."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    code = ("import sys, traceback; sys.path.insert(0, %r); from tests import host_checks\n"
            "for name in %r:\n"
            "    try:\n"
            "        getattr(host_checks, name)(); print('PASS', name)\n"
            "    except Exception:\n"
            "        print('FAIL', name); traceback.print_exc()\n") % (root, CHECKS)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    passed = [l.split()[1] for l in r.stdout.splitlines() if l.startswith("PASS ")]
    assert r.returncode == 0 and passed == CHECKS, r.stdout + r.stderr
