"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
and exports every function that include/nysadmm.h declares.  No compute call
is made here (there is no GPU on this host)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nysadmm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:nys_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2202_11599_gb300 import build_lib
    return build_lib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nys_sketch", "nys_precond_apply", "pcg_solve", "nysadmm_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_and_defaults_without_gpu(libpath):
    from paper_2202_11599_gb300 import nysadmm as nx
    assert nx.strerror(0) == "ok"
    assert "invalid" in nx.strerror(1)
    o = nx.NysOptsC()
    nx.lib().nys_opts_default(ctypes.byref(o))
    assert o.admm_maxit == 200 and o.refine == 1 and abs(o.ada_tol - 2.0) < 1e-15


def test_struct_layouts_match_header(libpath):
    from paper_2202_11599_gb300 import nysadmm as nx
    # offsets follow C natural alignment of the header's structs
    assert ctypes.sizeof(nx.NysMatrixC) == 48
    assert nx.NysOptsC.stream.offset == 96 and nx.NysOptsC.hx_refresh.offset == 108
    assert nx.NysOptsC.seed.offset == 128
    assert ctypes.sizeof(nx.NysOptsC) == 160
    assert ctypes.sizeof(nx.NysInfoC) == 48
    assert ctypes.sizeof(nx.NysStatsC) == 8 + 4 * 8 * 6


def test_invalid_arguments_rejected_before_any_launch(libpath):
    from paper_2202_11599_gb300 import nysadmm as nx
    L = nx.lib()
    # NULL matrix / bad shapes are rejected on the host, no CUDA call needed
    assert L.nys_hmatvec(None, None, 0.0, None, None, None) == nx.NYS_EINVAL
    m = nx.NysMatrixC(ctypes.c_void_p(16), nx.NYS_F64, 10, 0, 10)
    assert L.nys_hmatvec(ctypes.byref(m), None, 0.0, None, None, None) == nx.NYS_EINVAL
    m = nx.NysMatrixC(ctypes.c_void_p(16), nx.NYS_F64, 10, 5, 5)       # 5*8 bytes: not 16-aligned rows
    assert L.nys_hmatvec(ctypes.byref(m), None, 0.0, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == nx.NYS_EINVAL
    # FP8 storage needs its per-column scales, and scales belong to FP8 only
    m = nx.NysMatrixC(ctypes.c_void_p(16), nx.NYS_FP8E4M3, 10, 16, 16)
    assert L.nys_hmatvec(ctypes.byref(m), None, 0.0, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == nx.NYS_EINVAL
    m = nx.NysMatrixC(ctypes.c_void_p(16), nx.NYS_F32, 10, 16, 16, ctypes.c_void_p(64))
    assert L.nys_hmatvec(ctypes.byref(m), None, 0.0, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == nx.NYS_EINVAL


def test_elastic_net_gamma_range_checked_on_host(libpath):
    from paper_2202_11599_gb300 import nysadmm as nx
    L = nx.lib()
    m = nx.NysMatrixC(ctypes.c_void_p(16), nx.NYS_F64, 10, 16, 16)
    p = ctypes.c_void_p(64)
    for gamma in (0.0, -0.5, 1.5, float("nan")):
        # Eq. 6 needs 0 < gamma <= 1: rejected before any device work
        assert L.nysadmm_solve(nx.NYS_ELASTIC_NET, ctypes.byref(m), p, ctypes.c_double(gamma),
                               ctypes.c_double(1.0), 4, ctypes.c_double(1e-6), p, None, None, None,
                               None) == nx.NYS_EINVAL
        out = (ctypes.c_double * 3)()
        assert L.nys_objective(nx.NYS_ELASTIC_NET, ctypes.byref(m), p, ctypes.c_double(gamma), p,
                               out, None) == nx.NYS_EINVAL
    assert L.nysadmm_solve(7, ctypes.byref(m), p, ctypes.c_double(0.5), ctypes.c_double(1.0), 4,
                           ctypes.c_double(1e-6), p, None, None, None, None) == nx.NYS_EINVAL


def test_unknown_tolerance_mode_rejected_on_host(libpath):
    from paper_2202_11599_gb300 import nysadmm as nx
    L = nx.lib()
    m = nx.NysMatrixC(ctypes.c_void_p(16), nx.NYS_F64, 10, 16, 16)
    p = ctypes.c_void_p(64)
    o = nx.NysOptsC()
    L.nys_opts_default(ctypes.byref(o))
    o.pcg_tol_mode = 4
    assert L.nysadmm_solve(nx.NYS_LASSO, ctypes.byref(m), p, ctypes.c_double(0.5), ctypes.c_double(1.0), 4,
                           ctypes.c_double(1.0), p, ctypes.byref(o), None, None, None) == nx.NYS_EINVAL


def _header_enums():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    vals = {}
    for body in re.findall(r"typedef enum\s*\{(.*?)\}", src, flags=re.S):
        for name, v in re.findall(r"(\w+)\s*=\s*(-?\d+)", body):
            vals[name] = int(v)
    return vals


def test_binding_constants_match_header_enums():
    from paper_2202_11599_gb300 import nysadmm as nx
    h = _header_enums()
    for name in ("NYS_OK", "NYS_EINVAL", "NYS_ENOTSPD", "NYS_EBREAKDOWN", "NYS_ENOCONV", "NYS_ETIMEOUT",
                 "NYS_ECUDA", "NYS_ENOMEM", "NYS_LASSO", "NYS_LOGISTIC", "NYS_ELASTIC_NET", "NYS_F64",
                 "NYS_F32", "NYS_BF16", "NYS_FP8E4M3"):
        assert getattr(nx, name) == h[name], name
    modes = {"rel": "NYS_TOL_REL", "abs": "NYS_TOL_ABS", "sqrt_rprd": "NYS_TOL_SQRT_RPRD",
             "rnorm_pow": "NYS_TOL_RNORM_POW"}
    assert {k: h[v] for k, v in modes.items()} == nx.TOL_MODES


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof / offsetof of the header's structs from the C compiler equal the binding's."""
    import shutil
    import subprocess
    from paper_2202_11599_gb300 import nysadmm as nx
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in nx.NysOptsC._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nysadmm.h"', 'int main(void) {',
             'printf("%zu %zu %zu %zu\\n", sizeof(nys_matrix), sizeof(nys_opts), sizeof(nys_info), sizeof(nys_stats));']
    lines += [f'printf("%zu\\n", offsetof(nys_opts, {f}));' for f in fields]
    lines += ['return 0; }']
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    sizes = [int(v) for v in out[:4]]
    assert sizes == [ctypes.sizeof(nx.NysMatrixC), ctypes.sizeof(nx.NysOptsC), ctypes.sizeof(nx.NysInfoC),
                     ctypes.sizeof(nx.NysStatsC)]
    offs = [int(v) for v in out[4:]]
    assert offs == [getattr(nx.NysOptsC, f).offset for f in fields]
