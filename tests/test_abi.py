"""The C ABI library builds for sm_103a, loads, and exports every symbol include/qcd.h declares.

These run without a GPU: they make no compute call.  Argument checks that the
library performs before touching the device are exercised too.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libqcd():
    from paper_0910_0262_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qcd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(qcd_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("qcd_create", "qcd_destroy", "qcd_load_gauge", "qcd_clover_build", "qcd_dslash",
              "qcd_cg_solve", "qcd_fermion_force", "qcd_last_error"):
        assert n in names


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_compiles_on_its_own(tmp_path, compiler, std):
    """include/qcd.h is a plain C header: it compiles alone, as C99 and as C++, without warnings."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(compiler + " not found")
    src = tmp_path / "use_header.c"
    src.write_text('#include "qcd.h"\nint main(void) { return qcd_last_error() == 0; }\n')
    lang = ["-x", "c++"] if compiler == "g++" else []
    r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include")] + lang + [str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_every_declared_symbol_is_exported(libqcd):
    for n in declared_functions():
        assert hasattr(libqcd, n), n


def test_binding_names_match_the_abi():
    from paper_0910_0262_gb300 import qcd
    for n in declared_functions():
        assert n in qcd._SIGNATURES, n
        assert callable(getattr(qcd, n)), n


def test_create_rejects_bad_extents_without_a_device(libqcd):
    from paper_0910_0262_gb300 import qcd
    for dims in [(3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 5, 4)]:
        with pytest.raises(qcd.QCDError) as e:
            qcd.qcd_create(dims, -1.0, None)
        assert e.value.status == 1
        assert "even" in e.value.message
    with pytest.raises(qcd.QCDError) as e:
        qcd.qcd_create((4, 4, 4, 4), 0.5, None)
    assert e.value.status == 1


def test_null_context_is_an_argument_error(libqcd):
    from paper_0910_0262_gb300 import qcd
    L = qcd.lib()
    assert L.qcd_clover_build(None, 0.12, 1.0) == 1
    assert L.qcd_destroy(None) == 0
    assert "null" in qcd.qcd_last_error()


def test_extent_division_matches_integer_division(libqcd):
    """The kernels' multiply-and-shift division by X, Y, Z (host evaluation of the same expression)."""
    libqcd.qcd_selftest_fastdiv.restype = ctypes.c_longlong
    assert libqcd.qcd_selftest_fastdiv() == 0


def test_staged_block_order_is_a_permutation(libqcd):
    """The staged FP32 multi-RHS kernel's order of its 32-site blocks covers every block once (host
    evaluation of the same function, on every small even lattice and the benchmark lattices)."""
    libqcd.qcd_selftest_site_order.restype = ctypes.c_longlong
    assert libqcd.qcd_selftest_site_order() == 0


def test_local_group_host_calls(libqcd):
    """The in-process slab group's host-only calls: the group size is checked (1 to 16 slabs), and
    abort and destroy of a group that no slab joined touch no device."""
    from paper_0910_0262_gb300 import qcd as Q
    for n in (0, -1, 17):
        with pytest.raises(Q.QCDError) as e:
            Q.qcd_local_group_create(n)
        assert e.value.status == 1  # QCD_ERR_ARG
    g = Q.qcd_local_group_create(2)
    Q.qcd_local_group_abort(g)
    Q.qcd_local_group_destroy(g)
    assert libqcd.qcd_local_group_abort(None) == 1
    assert libqcd.qcd_local_group_destroy(None) == 0
