"""The C-ABI library builds, loads and exports every symbol include/flr.h declares, and
rejects bad parameters with a status code (CPU only: no call here reaches a kernel)."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2410_11625_gb300 import flr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return flr.load_library()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"flr_create", "flr_denoise", "flr_destroy"} <= names
    for name in names:
        assert hasattr(lib, name), name
    assert set(flr.EXPORTS) == names


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.flr_status_string(code)
    assert lib.flr_status_string(0) == b"FLR_OK"


@pytest.mark.parametrize("kw,status", [
    (dict(q=0), -4), (dict(q=9), -4), (dict(radius=17), -4), (dict(coef_radius=17), -4),
    (dict(radius=-1), -1), (dict(coef_radius=-1), -1), (dict(eps=-1.0), -1),
    (dict(eps=float("nan")), -1), (dict(flags=2), -1), (dict(pivot_ratio=float("nan")), -1),
])
def test_create_rejects_bad_params(lib, kw, status):
    p = dict(q=8, radius=8, coef_radius=8, eps=1e-3, pivot_ratio=1e-3, flags=0)
    p.update(kw)
    params = flr.FlrParams(p["q"], p["radius"], p["coef_radius"], p["eps"], p["pivot_ratio"], p["flags"])
    h = ctypes.c_void_p()
    assert lib.flr_create(ctypes.byref(params), ctypes.byref(h)) == status
    assert not h.value


@pytest.mark.parametrize("flags,eps_mul", [(0, 0.1), (flr.FLR_FAST_APPENDIX, 1.5), (flr.FLR_FAST_APPENDIX, -0.1),
                                           (2, 0.0), (flr.FLR_FAST_APPENDIX, float("nan"))])
def test_fast_create_rejects_bad_appendix_terms(lib, flags, eps_mul):
    """The Appendix flag and its multiplicative term (in [0, 1], 0 without the flag) are
    checked before any device work."""
    p = flr.FlrFastParams(8, 8, 1, 1.25, 3, 1e-3, 1e-3, flags, eps_mul)
    h = ctypes.c_void_p()
    assert lib.flr_fast_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.flr_create(None, None) == -1
    assert lib.flr_destroy(None) == 0
    assert lib.flr_denoise(None, None, None, None, None, 8, 8, None) == -1
    assert lib.flr_denoise_host(None, None, None, None, None, 8, 8, None) == -1
    assert lib.flr_denoise_host_async(None, None, None, None, None, 8, 8, None) == -1
    assert lib.flr_host_wait(None) == -1
    assert lib.flr_reserve(None, 8, 8) == -1
    assert lib.flr_get_stats(None, None) == -1
    assert lib.flr_get_kernel_times(None, None, 0) == -1


@pytest.mark.parametrize("r,rc", [(8, 8), (8, 0), (5, 5), (16, 3), (0, 0), (2, 16)])
def test_host_band_plan_covers_every_row_once(lib, r, rc):
    """flr_denoise_host's bands (host arithmetic only): the input copies and the output
    bands each partition the rows; a band's models need only input rows already copied;
    its averaged outputs need only models of earlier or current bands (below c[k+1])."""
    from paper_2410_11625_gb300 import flr
    for H in (1, 96, 539, 540, 600, 1080, 1100, 1440, 2160, 4320):
        c, e, o = flr.host_band_plan(H, r, rc)
        K = len(c) - 1
        assert K == max(1, min(flr.HOST_MAX_BANDS, (H + 180) // 360))
        assert c[0] == 0 and c[K] == H and all(c[k] < c[k + 1] for k in range(K))
        assert all(c[k] % 4 == 0 for k in range(K))  # segment rows stay multiples of kB
        assert e[0] == 0 and e[K] == H and all(e[k] <= e[k + 1] for k in range(K))
        assert o[0] == 0 and o[K] == H and all(o[k] < o[k + 1] for k in range(K))
        for k in range(K):
            assert e[k + 1] >= min(H, c[k + 1] + r)   # inputs of band k's windows
            assert o[k + 1] <= e[k + 1]               # its map-guide rows
            if k + 1 < K:
                assert o[k + 1] + rc <= c[k + 1]      # averaging windows of its outputs
            if rc == 0:
                assert o[k] == c[k]
