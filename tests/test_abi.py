"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point declared in include/srtm.h, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2410_00627_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "srtm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+(srtm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_binding_symbols():
    assert header_functions() == sorted(api.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # two 4-int headers then pointers on LP64
    assert ctypes.sizeof(api.Problem) == 16 + 7 * 8 + 8 + 2 * 8   # + nu (padded), B, u
    assert ctypes.sizeof(api.Output) == 5 * 8
    assert ctypes.sizeof(api.Batch) == 16 + 16 + 9 * 8 + 8 + 2 * 8
    assert ctypes.sizeof(api.Tuning) == 40


def test_rejects_bad_arguments_without_gpu(lib):
    assert lib.srtm_smoother(None, 0, None, None, None) == -1
    bad = api.Problem(9, 1, 2, 3)  # nx out of range: rejected before any pointer is inspected
    assert lib.srtm_smoother(ctypes.byref(bad), 0, None, None, None) == -6
    assert "nx=9" in api.last_error_detail()
    bad = api.Problem(2, 5, 2, 3)
    assert lib.srtm_filter(ctypes.byref(bad), 0, None, None) == -6
    bad = api.Problem(2, 1, 0, 3)
    assert lib.srtm_smoother(ctypes.byref(bad), 0, None, None, None) == -1
    bad = api.Problem(2, 1, 2, 3)
    assert lib.srtm_smoother(ctypes.byref(bad), 7, None, None, None) == -1
    assert lib.srtm_selftest_wait(0, None) == -1            # polls out of range
    assert lib.srtm_selftest_wait(2000001, None) == -1
    bad = api.Problem(9, 1, 2, 3)
    assert lib.srtm_smoother_sequential(ctypes.byref(bad), 0, None, None, None) == -6


def test_tuning_validation_and_roundtrip(lib):
    t = api.Tuning(0, 0, 0, 0, 0)
    assert lib.srtm_get_tuning(4, 1, ctypes.byref(t)) == 0
    assert t.scan_groups * 16 == 128 and t.scan_elems >= 1 and t.recover_threads % 32 == 0
    assert t.lookback_window == 16 and t.setup_mode == 1
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(3, 0, 0))) == -1   # not a power of two
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(32, 0, 0))) == -1  # 32*16 lanes > 256
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 48))) == -1  # not a multiple of 32
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 256))) == -1  # above the block bound
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 33))) == -1  # window above 32
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, -1))) == -1
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 3))) == -1   # setup_mode
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 3))) == -1  # recover_split
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 0, 17))) == -1  # batch_chunks
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 0, 0, 4))) == -1  # chunk_recover_bps
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 0, 0, 0, 9))) == -1  # chunk_scan_bps
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 0, 0, 0, 0, 3))) == -1  # recover_form
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 0, -1))) == -1
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(4, 8, 64, 8))) == 0
    assert lib.srtm_get_tuning(4, 1, ctypes.byref(t)) == 0
    assert (t.scan_groups, t.scan_elems, t.recover_threads, t.lookback_window) == (4, 8, 64, 8)
    assert lib.srtm_set_tuning(4, 1, ctypes.byref(api.Tuning(0, 0, 0))) == 0
    assert lib.srtm_set_tuning(1, 0, ctypes.byref(api.Tuning(128, 0, 0))) == 0
    assert lib.srtm_set_tuning(1, 0, ctypes.byref(api.Tuning(0, 0, 0))) == 0


def test_autotune_rejects_bad_arguments_without_gpu(lib):
    assert lib.srtm_autotune(None, 1, None, 1, None, None, None) == -1
    bad = api.Problem(9, 1, 2, 3)
    assert lib.srtm_autotune(ctypes.byref(bad), 1, None, 1, None, None, None) == -6
    ok_dims = api.Problem(2, 1, 2, 3)
    assert lib.srtm_autotune(ctypes.byref(ok_dims), 5, None, 1, None, None, None) == -1
    assert lib.srtm_autotune_batch(None, 1, None, 1, None, None, None) == -1


def test_launch_counts(lib):
    assert lib.srtm_launches_per_call(1, 0) == 4
    assert lib.srtm_launches_per_call(0, 0) == 3
    assert lib.srtm_launches_per_call(1, 1) == 5


def test_error_codes_match_header():
    """Every SRTM_* status the header declares has the same value and name in the binding."""
    src = open(os.path.join(ROOT, "include", "srtm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    codes = {int(v): k for k, v in re.findall(r"\b(SRTM_(?:OK|ERR_\w+))\s*=\s*(-?\d+)", src)}
    assert codes == api.ERRORS


def test_header_compiles_as_c99_and_links(lib, tmp_path):
    """A plain C99 program (gcc -pedantic -Werror, no CUDA headers) includes
    the header, links the library and checks the calls that need no GPU."""
    import subprocess
    libdir = os.path.join(ROOT, "paper_2410_00627_gb300")
    exe = str(tmp_path / "abi_c_check")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "abi_c_check.c"), "-o", exe, "-L", libdir, "-lsrtm",
                    "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == "ok"


@pytest.mark.parametrize("nx", range(1, 9))
def test_built_in_tunings_are_in_their_documented_ranges(lib, nx):
    lanes = {1: 1, 2: 4}.get(nx, 16 if nx <= 4 else 32)
    for prec in (0, 1, 2):
        t = api.Tuning(0, 0, 0, 0, 0, 0)
        assert lib.srtm_get_tuning(nx, prec, ctypes.byref(t)) == 0
        g = t.scan_groups
        assert g & (g - 1) == 0 and 32 <= g * lanes <= 256, (nx, prec, g)
        assert 1 <= t.scan_elems <= 64 and 32 <= t.recover_threads <= 128 and t.recover_threads % 32 == 0
        assert 1 <= t.lookback_window <= 32 and t.setup_mode in (1, 2) and t.recover_split in (1, 2)
        assert 1 <= t.batch_chunks <= 16 and 0 <= t.chunk_recover_bps <= 3 and 0 <= t.chunk_scan_bps <= 8
        assert t.recover_form in (1, 2)
        # every documented value of every field is accepted, one at a time, and read back
        for field, values in (("scan_elems", (1, 64)), ("recover_threads", (32, 128)),
                              ("lookback_window", (1, 32)), ("setup_mode", (1, 2)), ("recover_split", (1, 2)),
                              ("batch_chunks", (1, 16)), ("chunk_recover_bps", (1, 3)), ("chunk_scan_bps", (1, 8)),
                              ("recover_form", (1, 2))):
            for v in values:
                u = api.Tuning(0, 0, 0, 0, 0, 0)
                setattr(u, field, v)
                assert lib.srtm_set_tuning(nx, prec, ctypes.byref(u)) == 0, (nx, prec, field, v)
                back = api.Tuning(0, 0, 0, 0, 0, 0)
                assert lib.srtm_get_tuning(nx, prec, ctypes.byref(back)) == 0
                assert getattr(back, field) == v, (nx, prec, field, v)
        assert lib.srtm_set_tuning(nx, prec, ctypes.byref(api.Tuning(0, 0, 0, 0, 0, 0))) == 0   # built-in again


@pytest.mark.parametrize("nx", range(1, 9))
def test_scan_groups_bounds_follow_the_lanes_per_group(lib, nx):
    """scan_groups x lanes-per-group (1, 4, 16 or 32 by nx) must lie in 32..256."""
    lanes = {1: 1, 2: 4}.get(nx, 16 if nx <= 4 else 32)
    lo, hi = max(1, 32 // lanes), 256 // lanes
    assert lib.srtm_set_tuning(nx, 1, ctypes.byref(api.Tuning(lo, 0, 0))) == 0
    assert lib.srtm_set_tuning(nx, 1, ctypes.byref(api.Tuning(hi, 0, 0))) == 0
    assert lib.srtm_set_tuning(nx, 1, ctypes.byref(api.Tuning(hi * 2, 0, 0))) == -1
    if lo > 1:
        assert lib.srtm_set_tuning(nx, 1, ctypes.byref(api.Tuning(lo // 2, 0, 0))) == -1
    assert lib.srtm_set_tuning(nx, 1, ctypes.byref(api.Tuning(0, 0, 0))) == 0


def test_binding_rejects_non_cuda_inputs_before_any_call():
    """The binding marshals only contiguous CUDA float64 tensors (no CPU
    fallback): host tensors and numpy arrays are refused before the library
    is called; an unknown method is refused by name."""
    import numpy as np
    import torch
    F = torch.eye(2, dtype=torch.float64)
    args = [F, F, torch.ones(1, 2, dtype=torch.float64), torch.ones(1, 1, dtype=torch.float64),
            torch.zeros(2, dtype=torch.float64), F, torch.zeros(5, 1, dtype=torch.float64)]
    with pytest.raises(TypeError, match="CUDA float64"):
        api.smoother(*args, 3)
    with pytest.raises(TypeError, match="CUDA float64"):
        api.filter(*[a.numpy() for a in args], 3)
    with pytest.raises(ValueError, match="method"):
        api._entry("srtm_smoother", "bogus")
    assert np.isfinite(api.launches_per_call(True, False))


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libsrtm.so every call raises: there is no CPU fallback."""
    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api, "lib_path", lambda: str(tmp_path / "libsrtm.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.load()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.get_tuning(4, "mixed")
