"""The C ABI library builds, loads and exports every entry point that include/sipg.h declares.

No GPU needed: nothing here launches a kernel.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sipg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sipg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_01900_gb300 import build, native
    if not os.path.exists(native.LIB_PATH):
        build.build()
    return native.lib()


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for must in ("sipg_create", "sipg_operator_apply", "sipg_smooth", "sipg_vcycle", "sipg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1910_01900_gb300 import native
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(native.EXPORTS) == _declared()


def test_default_params_and_create_rejects_bad_input(lib):
    import ctypes
    from paper_1910_01900_gb300 import native
    p = native.Params()
    lib.sipg_default_params(ctypes.byref(p))
    assert (p.degree, p.cheb_degree, p.eig_iters) == (3, 5, 20)
    assert abs(p.cheb_lo - 0.06) < 1e-15 and abs(p.cheb_hi - 1.2) < 1e-15
    mesh = native.Mesh()
    h = ctypes.c_void_p()
    p.degree = 0   # invalid: rejected before any device work
    assert lib.sipg_create(ctypes.byref(mesh), ctypes.byref(p), ctypes.byref(h)) == native.EINVAL
    assert b"degree" in lib.sipg_last_error(None)


def test_product_package_has_no_cpu_fallback():
    # the package must not import the oracle anywhere
    pkg = os.path.join(ROOT, "paper_1910_01900_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("no CPU", ""), f
