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
    assert (p.degree, p.cheb_degree, p.eig_iters, p.fuse_tail) == (3, 5, 20, 1)
    assert abs(p.cheb_lo - 0.06) < 1e-15 and abs(p.cheb_hi - 1.2) < 1e-15
    mesh = native.Mesh()
    h = ctypes.c_void_p()
    p.degree = 0   # invalid: rejected before any device work
    assert lib.sipg_create(ctypes.byref(mesh), ctypes.byref(p), ctypes.byref(h)) == native.EINVAL
    assert b"degree" in lib.sipg_last_error(None)
    # a non-positive penalty would make the operator indefinite: refused at setup, as are other
    # out-of-range parameters and mesh descriptions
    good, _ = native.make_mesh(4)
    for field, value, word in (("penalty_factor", -1.0, b"penalty"), ("penalty_factor", 0.0, b"penalty"),
                               ("precision", 2, b"precision"), ("cheb_degree", 0, b"smoother"),
                               ("p_coarsen", 3, b"smoother"), ("coarse_solver", 2, b"coarse_solver"),
                               ("coarse_rtol", 0.0, b"coarse_rtol"), ("coarse_maxit", 0, b"coarse_maxit"),
                               ("fuse_tail", 2, b"fuse_tail")):
        q = native.Params()
        lib.sipg_default_params(ctypes.byref(q))
        setattr(q, field, value)
        assert lib.sipg_create(ctypes.byref(good), ctypes.byref(q), ctypes.byref(h)) == native.EINVAL, field
        assert word in lib.sipg_last_error(None), (field, lib.sipg_last_error(None))
    q = native.Params()
    lib.sipg_default_params(ctypes.byref(q))
    for field, value, word in (("bc", 2, b"bc"), ("m", 0, b"m must"), ("mapping_degree", 2, b"mapping")):
        bad, _ = native.make_mesh(4, deform=1)
        if field == "bc":
            bad.bc[3] = value
        elif field == "m":
            bad.m[1] = value
        else:
            bad.mapping_degree = value
        assert lib.sipg_create(ctypes.byref(bad), ctypes.byref(q), ctypes.byref(h)) == native.EINVAL, field
        assert word in lib.sipg_last_error(None), (field, lib.sipg_last_error(None))


def test_product_package_has_no_cpu_fallback():
    # the package must not import the oracle anywhere
    pkg = os.path.join(ROOT, "paper_1910_01900_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("no CPU", ""), f


def test_null_handles_and_bad_arguments_are_rejected_before_device_work(lib):
    """Every entry point answers SIPG_EINVAL to a null context, batch, mesh or output pointer
    (the error behaviour include/sipg.h states), without touching the device."""
    from paper_1910_01900_gb300 import native
    N = None
    calls = {
        "sipg_create": (N, N, N),
        "sipg_create_unstructured": (N, N, N),
        "sipg_destroy": (N,),
        "sipg_num_levels": (N, N),
        "sipg_num_dofs": (N, 0, N),
        "sipg_level_info": (N, 0, N, N, N),
        "sipg_lambda": (N, 1, N),
        "sipg_rhs": (N, 0, N),
        "sipg_l2_error": (N, 0, N, N),
        "sipg_operator_apply": (N, 0, N, N),
        "sipg_operator_apply_multi": (N, 0, 2, N, N),
        "sipg_level_apply": (N, 0, 0, N, N),
        "sipg_inverse_diagonal": (N, 1, 0, N),
        "sipg_smooth": (N, 1, N, N, 1),
        "sipg_restrict": (N, 1, N, N),
        "sipg_prolongate_add": (N, 1, N, N),
        "sipg_coarse_solve": (N, N, N),
        "sipg_coarse_info": (N, N, N, N, N),
        "sipg_coarse_amg_vcycle": (N, N, N),
        "sipg_vcycle": (N, N, N),
        "sipg_solve": (N, N, N, 1e-10, 10, 0, N),
        "sipg_solve_host": (N, N, N, 1e-10, 10, N),
        "sipg_solve_multi": (N, 2, N, N, 1e-10, 10, N),
        "sipg_time_apply": (N, 0, N, N, 1, N, N),
        "sipg_tile_shape": (N, 0, 0, 0, N),
        "sipg_set_tile_shape": (N, 0, 0, 0, 1),
        "sipg_smoother_train": (N, 100, 1, 0, N),
        "sipg_smoother_finetune": (N, 1, 0.0, N),
        "sipg_set_smoother": (N, 0, 0, 1),
        "sipg_mlp_shape": (N, N, N, N, N, N, N),
        "sipg_mlp_params": (N, 0, N),
        "sipg_mlp_forward": (N, N, 1, N),
        "sipg_mlp_gradients": (N, N, N, 1, N, N),
        "sipg_mlp_features": (N, N, N, N),
        "sipg_launch_count": (N,),
        "sipg_fma_peak": (2, N, N),
        "sipg_batch_create": (0, N, N, N),
        "sipg_batch_destroy": (N,),
        "sipg_batch_context": (N, 0, N),
        "sipg_batch_apply": (N, N, N),
        "sipg_batch_vcycle": (N, N, N),
        "sipg_batch_solve": (N, N, N, 1e-10, 10, N),
        "sipg_operator_apply_noalloc": (N, 3, 1.0, N, N, N),
    }
    skip = {"sipg_default_params", "sipg_last_error", "sipg_batch_last_error"}
    assert sorted(calls) == sorted(set(_declared()) - skip)
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == native.EINVAL, name


def test_header_is_plain_c_and_a_c_program_links_and_runs(lib, tmp_path):
    """include/sipg.h compiles as strict C99 (no C++ or framework types), and a C program linked
    against libsipg.so gets SIPG_EINVAL and the error text for a bad setup, with no GPU needed."""
    import shutil
    import subprocess
    from paper_1910_01900_gb300 import native
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_sipg.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "sipg.h"
int main(void) {
  sipg_mesh mesh;
  sipg_params prm;
  sipg_ctx *ctx = NULL;
  memset(&mesh, 0, sizeof mesh);
  sipg_default_params(&prm);
  for (int d = 0; d < 3; ++d) { mesh.m[d] = 4; mesh.lo[d] = 0.0; mesh.hi[d] = 1.0; }
  mesh.mapping_degree = 3;
  prm.degree = 9;                       /* out of range: refused before any device work */
  sipg_status st = sipg_create(&mesh, &prm, &ctx);
  printf("%d %s\n", (int)st, sipg_last_error(NULL));
  return (st == SIPG_EINVAL && ctx == NULL) ? 0 : 1;
}
''')
    exe = tmp_path / "use_sipg"
    libdir = os.path.dirname(native.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lsipg",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert r.stdout.startswith("%d " % native.EINVAL) and "degree" in r.stdout


def test_noalloc_apply_rejects_before_device_work(lib):
    """sipg_operator_apply_noalloc checks its arguments before touching a device: cell counts
    whose integer product would wrap (2^21 cells per axis), meshes beyond its static scratch,
    curved cells, and input and output ranges that overlap all give SIPG_EINVAL."""
    import ctypes
    from paper_1910_01900_gb300 import native

    def mesh(m, deform=0):
        ms = native.Mesh()
        for d in range(3):
            ms.m[d], ms.lo[d], ms.hi[d] = m, 0.0, 1.0
        ms.deform, ms.amp, ms.mapping_degree = deform, 0.1 if deform else 0.0, 3
        return ms

    buf = (ctypes.c_double * 2)()
    other = (ctypes.c_double * 2)()
    u, v = ctypes.cast(buf, ctypes.c_void_p), ctypes.cast(other, ctypes.c_void_p)
    for ms, deg, word in ((mesh(1 << 21), 1, b"64 MiB"), (mesh(64), 8, b"64 MiB"), (mesh(2, deform=1), 2, b"deform")):
        st = lib.sipg_operator_apply_noalloc(ctypes.byref(ms), deg, 1.0, u, v, None)
        assert st == native.EINVAL
        assert word in lib.sipg_last_error(None)
    # one cell of degree 1 has 8 values: v starting 4 values into u overlaps it
    one = mesh(1)
    st = lib.sipg_operator_apply_noalloc(ctypes.byref(one), 1, 1.0, u, ctypes.c_void_p(u.value + 32), None)
    assert st == native.EINVAL and b"overlap" in lib.sipg_last_error(None)
    st = lib.sipg_operator_apply_noalloc(ctypes.byref(one), 1, 1.0, u, u, None)
    assert st == native.EINVAL and b"overlap" in lib.sipg_last_error(None)


def test_unstructured_setup_rejects_bad_input_before_device_work(lib):
    """sipg_create_unstructured checks its parameters and mesh arrays before any device work:
    operator_only must be 1 (no multigrid hierarchy on unstructured meshes), vertex ids must be
    in range and face conditions 0 or 1."""
    import ctypes

    import numpy as np

    import sipg_inputs
    from paper_1910_01900_gb300 import native
    V, C, F, _, _ = sipg_inputs.scrambled_box((2, 1, 1), 3)
    V = np.ascontiguousarray(V, dtype=np.float64)

    def attempt(cells, face_bc, operator_only):
        Cc = np.ascontiguousarray(cells, dtype=np.int32)
        Fc = np.ascontiguousarray(face_bc, dtype=np.int32)
        hm = native.HexMesh()
        hm.nverts, hm.vertices, hm.ncells, hm.cells = len(V), V.ctypes.data, len(Cc), Cc.ctypes.data
        hm.face_bc = Fc.ctypes.data
        p = native.Params()
        lib.sipg_default_params(ctypes.byref(p))
        p.degree, p.operator_only = 2, operator_only
        h = ctypes.c_void_p()
        return lib.sipg_create_unstructured(ctypes.byref(hm), ctypes.byref(p), ctypes.byref(h))

    assert attempt(C, F, 0) == native.EINVAL and b"operator_only" in lib.sipg_last_error(None)
    bad = C.copy()
    bad[0, 5] = -1
    assert attempt(bad, F, 1) == native.EINVAL and b"vertex id" in lib.sipg_last_error(None)
    badf = F.copy()
    badf[1, 2] = 3
    assert attempt(C, badf, 1) == native.EINVAL and b"face_bc" in lib.sipg_last_error(None)
