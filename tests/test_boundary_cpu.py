"""The C-ABI library builds, loads and exports every entry point include/airg.h declares (no GPU
calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "airg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(airg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2408_08262_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("airg_setup", "airg_solve", "airg_free", "airg_cf_split"):
        assert required in names


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as C99 with no torch or C++ types
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "airg.h"\nint main(void) { airg_params p; airg_params_default(&p); return p.seed == 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                        "-o", str(tmp_path / "use.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_2408_08262_gb300 import airg
    assert sorted(airg.EXPORTED) == declared_functions()


def test_params_default_and_status_strings(libpath):
    from paper_2408_08262_gb300 import airg
    p = airg._Params()
    airg.lib().airg_params_default(ctypes.byref(p))
    assert p.strong_threshold == 0.5 and p.ddc_fraction == 0.1 and p.pmisr_max_loops == 3
    assert p.drop_R == 0.01 and p.drop_Ac == 0.001 and p.n_smooth_up == 2 and p.coarse_poly_order == 12
    assert p.seed == 240808262
    # Python defaults mirror the C defaults
    d = airg.Params()
    for k, _ in airg._Params._fields_:
        assert getattr(p, k) == getattr(d, k), k
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert airg.lib().airg_status_string(code)


def test_setup_rejects_null_arguments_without_gpu(libpath):
    from paper_2408_08262_gb300 import airg
    out = ctypes.c_void_p()
    assert airg.lib().airg_setup(None, None, None, ctypes.byref(out)) == -1
    assert airg.lib().airg_solve(None, None, None, None, None, None) == -1


def test_parameter_and_argument_checks_run_before_any_device_work(libpath):
    # the variants' parameter rules and the new entry points' argument checks are host-side: they
    # reject before the library touches the device (the CSR pointers below are never dereferenced)
    from paper_2408_08262_gb300 import airg
    L = airg.lib()
    A = airg._Csr(8, 8, 16, 32, 48)  # n, nnz, non-null stand-in pointers
    out = ctypes.c_void_p()

    def setup(**kw):
        p = airg.Params(**kw).c()
        return L.airg_setup(ctypes.byref(A), ctypes.byref(p), None, ctypes.byref(out))

    for bad in (dict(matrix_free=2), dict(matrix_free=1, precision=1), dict(matrix_free=1, precision=2),
                dict(ideal_prolong=3), dict(ideal_prolong=1, precision=1), dict(sparsity_order=3),
                dict(sparsity_order=0), dict(poly_order=15), dict(coarse_iters=0), dict(strong_threshold=1.5),
                dict(ddc_fraction=-0.1), dict(precision=7)):
        assert setup(**bad) == -1, bad
        assert out.value is None
    p = airg.Params().c()
    assert L.airg_setup_reuse(ctypes.byref(A), ctypes.byref(p), None, 0, None, ctypes.byref(out)) == -1
    assert L.airg_ddc_theta(None, None, None, None) == -1
    assert L.airg_ddc_theta(ctypes.byref(A), None, None, None) == -1
    assert L.airg_batch_tuned(None, None, None, 0) == -1
    # the entry point without allocation takes airg_cf_split's argument checks, before its capacity
    # check and before any device work
    cfo = ctypes.c_void_p(64)
    for bad in (dict(poly_order=15), dict(coarse_iters=0), dict(strong_threshold=1.5), dict(precision=7),
                dict(matrix_free=2), dict(sparsity_order=3)):
        p = airg.Params(**bad).c()
        assert L.airg_cf_split_noalloc(ctypes.byref(A), ctypes.byref(p), 0, cfo, None) == -1, bad
        assert L.airg_cf_split(ctypes.byref(A), ctypes.byref(p), 0, cfo, None) == -1, bad
    p = airg.Params().c()
    assert L.airg_cf_split_noalloc(None, ctypes.byref(p), 0, cfo, None) == -1
    assert L.airg_cf_split_noalloc(ctypes.byref(A), None, 0, cfo, None) == -1
    assert L.airg_cf_split_noalloc(ctypes.byref(A), ctypes.byref(p), 0, None, None) == -1
    assert L.airg_cf_split_noalloc(ctypes.byref(A), ctypes.byref(p), -1, cfo, None) == -1
    Anull = airg._Csr(8, 8, None, 32, 48)
    assert L.airg_cf_split_noalloc(ctypes.byref(Anull), ctypes.byref(p), 0, cfo, None) == -1
    # beyond the fixed array: rejected with its own code, still before any device work
    Abig = airg._Csr(10_000_000, 100_000_000, 16, 32, 48)
    assert L.airg_cf_split_noalloc(ctypes.byref(Abig), ctypes.byref(p), 0, cfo, None) == -8


def test_host_setup_checks_its_arguments_before_any_device_work(libpath):
    # airg_setup_host takes airg_setup's argument and parameter checks (host-side)
    from paper_2408_08262_gb300 import airg
    L = airg.lib()
    out = ctypes.c_void_p()
    p = airg.Params().c()
    assert L.airg_setup_host(None, ctypes.byref(p), None, ctypes.byref(out)) == -1
    A = airg._Csr(8, 8, 16, 32, 48)
    assert L.airg_setup_host(ctypes.byref(A), None, None, ctypes.byref(out)) == -1
    bad = airg.Params(poly_order=15).c()
    assert L.airg_setup_host(ctypes.byref(A), ctypes.byref(bad), None, ctypes.byref(out)) == -1
    assert L.airg_setup_host(ctypes.byref(A), ctypes.byref(p), None, None) == -1
    assert out.value is None


def test_concurrent_setups_check_their_arguments_before_any_device_work(libpath):
    from paper_2408_08262_gb300 import airg
    L = airg.lib()
    p = airg.Params().c()
    outs = (ctypes.c_void_p * 2)()
    As = (airg._Csr * 2)(airg._Csr(8, 8, 16, 32, 48), airg._Csr(8, 8, None, 32, 48))
    assert L.airg_setup_many(None, 2, ctypes.byref(p), 2, None, outs) == -1
    assert L.airg_setup_many(As, 0, ctypes.byref(p), 2, None, outs) == -1
    assert L.airg_setup_many(As, 2, ctypes.byref(p), 2, None, outs) == -1  # second CSR has no row pointers
    bad = airg.Params(coarse_iters=0).c()
    assert L.airg_setup_many(As, 1, ctypes.byref(bad), 2, None, outs) == -1
    assert L.airg_setup_many(As, 1, ctypes.byref(p), 2, None, None) == -1
    assert outs[0] is None and outs[1] is None
