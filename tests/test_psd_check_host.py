"""The covariance check behind SRTM_ERR_NOT_PSD, compiled for the host and
tested against numpy's eigenvalues: it must accept every symmetric positive
semi-definite matrix (singular ones included, and rounding-level asymmetry)
and reject clearly indefinite, asymmetric or non-finite ones, for n = 1..8."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2410_00627_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def check(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("psd") / "libpsd.so")
    cmd = [build._nvcc(), *build.ARCH, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I" + build.CSRC, "-I" + build.INCLUDE, os.path.join(HERE, "native", "psd_check_host.cu"), "-o", so]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    lib.psd_check_host.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]

    def f(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return bool(lib.psd_check_host(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.shape[0]))
    return f


def _psd(rng, n, rank, scale=1.0):
    G = rng.standard_normal((n, rank))
    return scale * G @ G.T


@pytest.mark.parametrize("n", range(1, 9))
def test_accepts_positive_semidefinite(check, n):
    rng = np.random.default_rng(n)
    for rank in range(0, n + 1):
        for scale in (1e-8, 1.0, 1e6):
            a = _psd(rng, n, rank, scale)
            a = 0.5 * (a + a.T)
            assert check(a), (n, rank, scale)
    a = _psd(rng, n, n)
    b = a.copy()
    b[0, -1] += 1e-13 * np.max(np.diag(a))   # asymmetric to rounding
    assert check(b)


@pytest.mark.parametrize("n", range(1, 9))
def test_rejects_indefinite(check, n):
    rng = np.random.default_rng(100 + n)
    for trial in range(20):
        V, _ = np.linalg.qr(rng.standard_normal((n, n)))
        ev = rng.uniform(0.1, 1.0, n)
        ev[rng.integers(n)] = -rng.choice([1e-3, 1e-1, 1.0])
        a = (V * ev) @ V.T
        a = 0.5 * (a + a.T)
        assert np.linalg.eigvalsh(a)[0] < -1e-4
        assert not check(a), (n, trial)


@pytest.mark.parametrize("n", range(2, 9))
def test_rejects_indefinite_behind_a_zero_pivot(check, n):
    """A zero diagonal entry with a non-zero off-diagonal in its row: a 2 x 2
    principal minor is negative, whatever the rest."""
    a = np.eye(n)
    a[0, 0] = 0.0
    a[0, n - 1] = a[n - 1, 0] = 1e-3
    assert np.linalg.eigvalsh(a)[0] < 0
    assert not check(a)


@pytest.mark.parametrize("n", range(2, 9))
def test_rejects_asymmetric_and_non_finite(check, n):
    rng = np.random.default_rng(200 + n)
    a = _psd(rng, n, n)
    s = np.max(np.diag(a))
    b = a.copy()
    b[n - 1, 0] += 1e-6 * s
    assert not check(b)
    for bad in (np.nan, np.inf, -np.inf):
        c = a.copy()
        c[1, 0] = c[0, 1] = bad
        assert not check(c)
        c = a.copy()
        c[n - 1, n - 1] = bad
        assert not check(c)
