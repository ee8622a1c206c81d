"""The C-ABI boundary without a GPU: libpff builds and loads, exports every entry point that
include/pff.h declares, the Python binding knows each of them, the host-only entry points behave as
documented, argument checks fail before any CUDA work, and the binding refuses to run without the
library (there is no fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "pff.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*|long long)\s+(pff_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_00331_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared()
    for required in ("pff_setup_mesh", "pff_set_state", "pff_apply_jacobian", "pff_residual", "pff_vcycle",
                     "pff_solve_newton_step", "pff_param_grad", "pff_destroy", "pff_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_the_header():
    from paper_2005_00331_gb300 import pff
    assert set(declared()) <= set(pff._SIGS)


def test_host_entry_points(lib):
    from paper_2005_00331_gb300 import pff
    p = pff.Params()
    lib.pff_default_params(ctypes.byref(p))
    assert (p.dim, p.degree, p.coarse_min, p.cheb_degree, p.eig_iters, p.gmres_restart) == (2, 1, 3, 5, 15, 50)
    assert abs(p.cheb_lo - 0.24) < 1e-15 and abs(p.cheb_hi - 1.2) < 1e-15 and abs(p.lin_rtol - 1e-6) < 1e-20
    lib.pff_strerror.restype = ctypes.c_char_p
    assert lib.pff_strerror(0) == b"ok"
    assert lib.pff_strerror(-1) == b"invalid argument"
    lib.pff_launch_count.restype = ctypes.c_longlong
    assert lib.pff_launch_count() >= 0


@pytest.mark.parametrize("field,value", [("dim", 4), ("degree", 0), ("degree", 9), ("n_cells_1d", 0),
                                         ("mg_precision", 16), ("cheb_degree", 0), ("eig_iters", 65),
                                         ("gmres_restart", 0), ("lin_rtol", 0.0), ("eps", -1.0), ("fp64_mode", 2)])
def test_setup_rejects_bad_parameters_before_cuda(lib, field, value):
    from paper_2005_00331_gb300 import pff
    p = pff.Params()
    lib.pff_default_params(ctypes.byref(p))
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.pff_setup_mesh(ctypes.byref(h), ctypes.byref(p), None) == -1
    assert not h.value


@pytest.mark.parametrize("dim,degree,cells", [(2, 2, 18920), (2, 4, 30000), (3, 1, 1290), (3, 2, 1 << 21)])
def test_setup_rejects_more_dofs_than_32bit_indices(lib, dim, degree, cells):
    # 3 (2p N + 1)^2 or 4 (p N + 1)^3 DoFs above 2^31 - 1: TOO_LARGE before any CUDA call
    from paper_2005_00331_gb300 import pff
    p = pff.Params()
    lib.pff_default_params(ctypes.byref(p))
    p.dim, p.degree, p.n_cells_1d = dim, degree, cells
    h = ctypes.c_void_p()
    assert lib.pff_setup_mesh(ctypes.byref(h), ctypes.byref(p), None) == -8
    assert not h.value


def test_null_context_is_rejected(lib):
    n = ctypes.c_longlong()
    i = ctypes.c_int()
    assert lib.pff_sizes(None, ctypes.byref(n), ctypes.byref(n), ctypes.byref(i)) == -1
    assert lib.pff_residual(None, None) == -1
    assert lib.pff_vcycle(None, None, None) == -1
    assert lib.pff_apply_jacobian(None, 0, None, None, 64, 0) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2005_00331_gb300 import pff
    monkeypatch.setattr(pff, "_LIB", None)
    monkeypatch.setattr(pff, "library_path", lambda: str(tmp_path / "libpff.so"))
    with pytest.raises(RuntimeError):
        pff.load_library(build_if_missing=False)


def test_plain_c_consumer(lib, tmp_path):
    """include/pff.h compiles as strict C99, and a C program linked against libpff
    (tests/abi_consumer.c) runs the host-only entry points and gets the documented results."""
    import shutil
    import subprocess
    from paper_2005_00331_gb300 import build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    libdir = os.path.dirname(build.build())
    exe = str(tmp_path / "abi_consumer")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "abi_consumer.c"), "-o", exe, "-L", libdir, "-lpff",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    lines = r.stdout.strip().splitlines()
    assert r.returncode == 0 and lines[-1] == "ok", (r.returncode, r.stdout, r.stderr)
    # the binding's ctypes mirror of pff_params has the C layout
    import ctypes
    from paper_2005_00331_gb300.pff import Params
    size, off_fp64, off_coarse, off_slit = (int(v) for v in lines[0].split()[1:])
    assert ctypes.sizeof(Params) == size
    assert (Params.fp64_mode.offset, Params.coarse_precision.offset, Params.slit_cut.offset) == \
        (off_fp64, off_coarse, off_slit)


def test_status_codes_match_the_header():
    """The binding's PFF_OK / PFF_ERR_* constants are the header's values, and every code has a message."""
    import paper_2005_00331_gb300 as pkg
    src = open(os.path.join(ROOT, "include", "pff.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"#define (PFF_(?:OK|ERR_\w+))\s+\(?(-?\d+)\)?", src))
    assert len(codes) >= 10
    for name, value in codes.items():
        assert getattr(pkg, name) == value, name
    lib = pkg.load_library()
    for name, value in codes.items():
        if value:
            assert lib.pff_strerror(value).decode() != "unknown status", name
