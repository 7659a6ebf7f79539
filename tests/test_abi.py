"""The C ABI library loads without a GPU and exports every function include/fdbem.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fdbem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_1311_5202_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("bm_problem_create", "fda_build_tree", "fda_tree_export", "fda_precompute_translations",
              "fda_matvec", "bm_gmres_solve", "bm_rhs_plane_wave", "fda_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds_without_gpu(built):
    from paper_1311_5202_gb300 import fdbem
    L = fdbem.lib()
    for n in _declared():
        assert hasattr(L, n)
    assert fdbem.fda_last_error() == ""


def test_binding_signature_table_covers_header():
    from paper_1311_5202_gb300 import fdbem
    assert sorted(n for n, _, _ in fdbem._SIGS) == _declared()


def test_invalid_arguments_fail_cleanly_without_gpu(built):
    """Argument checks run before any device work and return FDA_E_INVALID_ARG with a message."""
    import ctypes as C

    import numpy as np

    from paper_1311_5202_gb300 import fdbem
    h = C.c_void_p()
    nodes = np.zeros((3, 3))
    elems = np.zeros((0, 6), dtype=np.int32)
    rc = fdbem.lib().bm_problem_create(fdbem._ptr(nodes), 3, fdbem._ptr(elems, C.c_int32), 0, 1.0, 0.0, 1.0,
                                       C.byref(h))
    assert rc == fdbem.FDA_E_INVALID_ARG
    assert "empty" in fdbem.fda_last_error()
    rc = fdbem.lib().bm_problem_create(fdbem._ptr(nodes), 3, fdbem._ptr(elems, C.c_int32), 1, -1.0, 0.0, 1.0,
                                       C.byref(h))
    assert rc == fdbem.FDA_E_INVALID_ARG
    cfg = fdbem.fda_config_t()
    cfg.eps = 2.0
    rc = fdbem.lib().fda_precompute_translations(None, C.byref(cfg), C.byref(h))
    assert rc == fdbem.FDA_E_INVALID_ARG and "eps" in fdbem.fda_last_error()
    # configuration fields are checked before the tree
    cfg.eps, cfg.precision, cfg.nrhs_max = 1e-4, fdbem.FDA_PREC_FP32, 1
    for field, bad, word in (("m2l_tensor", 4, "m2l_tensor"), ("op", 3, "op"), ("near_split", 3, "near_split"),
                             ("drop_fp64", 2, "drop_fp64"), ("near_form", 5, "near_form"),
                             ("nrhs_max", 0, "nrhs_max")):
        good = getattr(cfg, field)
        setattr(cfg, field, bad)
        rc = fdbem.lib().fda_precompute_translations(None, C.byref(cfg), C.byref(h))
        assert rc == fdbem.FDA_E_INVALID_ARG and word in fdbem.fda_last_error(), field
        setattr(cfg, field, good)
    rc = fdbem.lib().fda_precompute_translations(None, C.byref(cfg), C.byref(h))
    assert rc == fdbem.FDA_E_INVALID_ARG and "tree" in fdbem.fda_last_error()
    # product schedule and precision checks come before the plan is touched
    assert fdbem.lib().fda_overlap_force(None, 1, 0, 0) == fdbem.FDA_E_INVALID_ARG
    assert "NULL plan" in fdbem.fda_last_error()
    x = (C.c_double * 4)()
    rc = fdbem.lib().fda_matvec_ex(None, fdbem.FDA_PREC_TF32, x, x, 1, fdbem.FDA_CPLX64, None)
    assert rc == fdbem.FDA_E_INVALID_ARG and "NULL" in fdbem.fda_last_error()


def test_struct_layouts_match_the_binding(tmp_path):
    """Every struct the header declares has the same size and field offsets in the ctypes binding (gcc compiles
    a probe against include/fdbem.h; no GPU)."""
    import ctypes as C

    from paper_1311_5202_gb300 import fdbem
    structs = [fdbem.fda_config_t, fdbem.bm_gmres_opts_t, fdbem.bm_gmres_stats_t, fdbem.fda_tree_view_t,
               fdbem.fda_tune_report_t, fdbem.fda_plan_info_t]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fdbem.h"', "int main(void) {"]
    for S in structs:
        n = S.__name__
        lines.append(f'  printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        n, f, v = line.split()
        got[(n, f)] = int(v)
    for S in structs:
        n = S.__name__
        assert got[(n, "size")] == C.sizeof(S), n
        for f, _ in S._fields_:
            assert got[(n, f)] == getattr(S, f).offset, (n, f)
