"""Host functions of the library (no device work): false-alarm probability of a
threshold over independent cells, its inverse, and the cell count, against the
oracle.  Runs without a GPU."""
import numpy as np
import pytest

from oracle import fstat as ofs


@pytest.fixture(scope="module")
def fs():
    from paper_1003_0844_gb300 import build, fstat
    build.build()
    fstat.load_library()
    return fstat


@pytest.mark.parametrize("F0,nc", [(0.0, 1.0), (3.0, 1.0), (20.0, 4.3e6), (31.5, 1e12), (60.0, 1e9)])
def test_false_alarm_matches_oracle(fs, F0, nc):
    a, nf = fs.false_alarm(F0, nc)
    ra, rnf = ofs.search_false_alarm(F0, nc)
    assert abs(a - ra) <= 1e-13 * max(ra, 1e-300) + 1e-300
    assert abs(nf - rnf) <= 1e-13 * max(rnf, 1e-300)
    assert fs.load_library().fs_false_alarm_cell(F0) == pytest.approx(float(ofs.false_alarm_probability(F0)),
                                                                      rel=1e-14)


@pytest.mark.parametrize("alpha,nc", [(0.01, 1e9), (1e-3, 4.3e6), (0.5, 10.0), (1e-6, 1.0), (0.9, 1e3)])
def test_threshold_inverts_the_false_alarm(fs, alpha, nc):
    F0 = fs.threshold(alpha, nc)
    assert F0 == pytest.approx(ofs.threshold_for_false_alarm(alpha, nc), rel=1e-10)
    assert fs.false_alarm(F0, nc)[0] == pytest.approx(alpha, rel=1e-9)


def test_threshold_and_count_errors(fs):
    with pytest.raises(fs.FstatError):
        fs.threshold(0.0, 10.0)
    with pytest.raises(fs.FstatError):
        fs.threshold(0.5, -1.0)
    with pytest.raises(fs.FstatError):
        fs.cell_count(np.array([[1.0, 2.0], [2.0, 1.0]]), 1.0)     # not positive definite


def test_cell_count_matches_oracle(fs):
    for G in (np.array([[1 / 12, 1 / 12], [1 / 12, 4 / 45]]),
              np.array([[3.0, 0.4, 0.1, 0.0], [0.4, 2.0, 0.2, 0.1], [0.1, 0.2, 1.5, 0.3], [0.0, 0.1, 0.3, 1.0]])):
        assert fs.cell_count(G, 123.0) == pytest.approx(ofs.cell_count(G, 123.0), rel=1e-12)
