"""Host side of the FFT search of the constrained lattice: the library's
fs_lattice_templates against the oracle's lattice_templates (sky positions,
spindown rows, bin offsets, padding), the size query and the argument rules."""
import math

import numpy as np
import pytest

from oracle import grid as og
from paper_1003_0844_gb300 import workloads as W


@pytest.fixture(scope="module")
def fs():
    from paper_1003_0844_gb300 import build, fstat
    build.build()
    fstat.load_library()
    return fstat


def _basis(name):
    wl = W.WORKLOADS[name]
    det = W.detector_for(wl)
    G = og.linear_model_fisher(wl.n, wl.dt, det)
    B, _, _ = og.constrained_lattice(G, 0.75, 2 * math.pi / (wl.nfft * wl.dt))
    return wl, det, B


@pytest.mark.parametrize("name,box,f1r", [("small", (0.30, 0.45, -0.10, 0.05), (-2e-9, 0.0)),
                                          ("tiny", None, (-1e-8, 0.0))])
def test_templates_match_oracle(fs, name, box, f1r):
    wl, det, B = _basis(name)
    a, d, f1, off = fs.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, f1r, box)
    T = og.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, *f1r, **({"box": box} if box else {}))
    assert len(a) == len(T) > 0
    nspin = f1.shape[1]
    assert nspin == max(len(r) for _, _, r in T)
    for i, (al, de, rows) in enumerate(T):
        assert abs(a[i] - al) <= 1e-12 and abs(d[i] - de) <= 1e-12
        for j in range(nspin):
            fr, dr, _ = rows[min(j, len(rows) - 1)]     # padded with the row's last node
            assert abs(f1[i, j] - fr) <= 1e-24 and abs(off[i, j] - dr) <= 1e-9
    assert np.all((off >= 0) & (off < 1))


def test_size_query_and_capacity(fs):
    import ctypes
    wl, det, B = _basis("tiny")
    lib = fs.load_library()
    b = np.ascontiguousarray(B)
    dd = fs._Detector(det.lat, det.lon, det.gamma, det.eps, det.lambda_e0, det.theta_g0)
    ns, nm = ctypes.c_int64(), ctypes.c_int32()
    args = (b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(dd), wl.fl, wl.nfft, wl.dt, -1e-8, 0.0,
            None)
    assert lib.fs_lattice_templates(*args, None, None, None, None, 0, 0, ctypes.byref(ns), ctypes.byref(nm)) == 0
    assert ns.value > 10 and nm.value > 1
    buf = [np.empty(ns.value * nm.value) for _ in range(4)]
    p = [x.ctypes.data_as(ctypes.c_void_p) for x in buf]
    st = lib.fs_lattice_templates(*args, *p, ns.value - 1, nm.value, ctypes.byref(ns), ctypes.byref(nm))
    assert st == 3   # FS_ERR_CAPACITY
    # a0 not on this transform's Fourier spacing
    with pytest.raises(fs.FstatError) as e:
        fs.lattice_templates(B, det, wl.fl, 2 * wl.nfft, wl.dt, (-1e-8, 0.0))
    assert e.value.status == 1
