"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares.  No compute call: this runs without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"FS_API\s+[\w\s\*]*?\b(fs_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1003_0844_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared_symbols()
    for must in ("fs_create", "fs_prepare_segment", "fs_search", "fs_sync_status", "fs_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    """The binding's list of entry points is exactly the header's declarations."""
    from paper_1003_0844_gb300 import fstat
    assert sorted(fstat.EXPORTS) == _declared_symbols()


def test_header_is_plain_c(tmp_path):
    """include/fstat.h compiles as strict C99 on its own (no CUDA or C++ headers)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "fstat.h"\nint main(void) { return fs_strerror(0) == 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_host_entry_points(lib, tmp_path):
    """A plain C program links against libfstat.so and calls host-only entry points:
    the false-alarm probability of Eqs. PF, FP, 1 - (1 - (1 + F0) exp(-F0))^n, and its
    inverse, against the closed form."""
    import math
    import shutil
    import subprocess
    from paper_1003_0844_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(build.build())
    src = tmp_path / "use_lib.c"
    src.write_text(
        '#include <stdio.h>\n#include "fstat.h"\n'
        'int main(void) {\n'
        '  double pf = 0.0, nf = 0.0, thr = 0.0;\n'
        '  if (fs_false_alarm(20.0, 1e6, &pf, &nf) != FS_OK) return 1;\n'
        '  if (fs_threshold(0.01, 1e6, &thr) != FS_OK) return 2;\n'
        '  printf("%.17g %.17g %.17g\\n", pf, nf, thr);\n'
        '  return 0;\n}\n')
    exe = str(tmp_path / "use_lib")
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lfstat",
                        "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    pf, nf, thr = map(float, r.stdout.split())
    cell = 21.0 * math.exp(-20.0)
    assert pf == pytest.approx(-math.expm1(1e6 * math.log1p(-cell)), rel=1e-12)
    assert nf == pytest.approx(1e6 * cell, rel=1e-12)
    back = -math.expm1(1e6 * math.log1p(-(1.0 + thr) * math.exp(-thr)))
    assert back == pytest.approx(0.01, rel=1e-9)


def test_strerror_is_host_only(lib):
    lib.fs_strerror.restype = ctypes.c_char_p
    assert lib.fs_strerror(0) == b"ok"
    assert lib.fs_strerror(3) == b"candidate buffer overflow"


def test_null_arguments_rejected_without_device(lib):
    # argument errors are returned before any CUDA call
    assert lib.fs_create(None, None, 0) == 1
    assert lib.fs_search(None, None, None, None, 0, None, 0, ctypes.c_float(0), None, ctypes.c_int64(0), None,
                         ctypes.c_int64(0), None, None) == 1
    assert lib.fs_search_noalloc(None, None, None, None, 0, None, 0, ctypes.c_float(0), None, ctypes.c_int64(0),
                                 None, ctypes.c_int64(0), None, None) == 1
    assert lib.fs_search_lattice_batch(None, None, 0, None, None, None, None, None, None, ctypes.c_float(0), None,
                                       ctypes.c_int64(0), None, None) == 1
    for name in ("fs_search_lattice", "fs_search_lattice_noalloc"):
        assert getattr(lib, name)(None, None, None, None, 0, None, None, 0, ctypes.c_float(0), None,
                                  ctypes.c_int64(0), None, ctypes.c_int64(0), None, None) == 1, name


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1003_0844_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f


def test_adjoint_entry_points_refuse_null_arguments(lib):
    """The adjoint's entry points check their arguments before any device call:
    null handles or pointers and empty point lists return FS_ERR_ARG."""
    vp = ctypes.c_void_p
    lib.fs_fstat_resampled.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp]
    lib.fs_fstat_resampled_grad.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp]
    lib.fs_refine_resampled.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
    for f in (lib.fs_fstat_resampled, lib.fs_fstat_resampled_grad, lib.fs_refine_resampled):
        f.restype = ctypes.c_int
    FS_ERR_ARG = 1
    assert lib.fs_fstat_resampled(None, None, None, 1, None, None) == FS_ERR_ARG
    assert lib.fs_fstat_resampled_grad(None, None, None, 1, None, None, None, None) == FS_ERR_ARG
    assert lib.fs_refine_resampled(None, None, None, 1, 20, None, None) == FS_ERR_ARG
