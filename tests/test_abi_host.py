"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/psa.h declares, sizes its workspace as documented and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2605_04550_gb300 import _native
from paper_2605_04550_gb300.build import ROOT, build_library

HEADER = os.path.join(ROOT, "include", "psa.h")


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _native.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psa_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert _declared_functions() == sorted(_native.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_version_and_strerror(lib):
    assert lib.psa_version() >= 100
    for code in (0, -1, -2, -3, -4):
        assert lib.psa_strerror(code)
    assert b"unsupported" in lib.psa_strerror(-4)


def test_default_opts(lib):
    o = lib.psa_default_opts()
    assert (o.k_min, o.k_max, o.tol, o.seed) == (2, 1000, 1e-13, 0)


def _ws(lib, n, kl, ku, P, kmax=1000, npoints=0):
    out = ctypes.c_size_t()
    o = _native.PsaLanczosOpts(2, kmax, 1e-13, 0)
    rc = lib.psa_workspace_bytes(ctypes.byref(_native.PsaBand(n, kl, ku, None)), ctypes.byref(o), P, npoints,
                                 ctypes.byref(out))
    return rc, out.value


def test_workspace_bytes_layout(lib):
    rc, b = _ws(lib, 2000, 2, 5, 128)
    assert rc == 0
    n, S, P, kmax = 2000, 10, 128, 1000
    # per point: factor (S complex) + 3 vectors + pivot byte per row, 2 k_max doubles
    per_point = 16 * n * S + 3 * 16 * n + n + 2 * 8 * kmax
    expect = per_point * P + 16 * n + 256
    # row records are padded to 512-byte fields plus a 128-byte pivot slot per warp
    assert expect <= b <= expect + (P // 32) * (n * (128 - 32) + 256) + 256
    # rounded up to whole warps
    assert _ws(lib, 2000, 2, 5, 97)[1] == _ws(lib, 2000, 2, 5, 128)[1]
    # the work-order schedule: 32 KB (histogram and cursors of 4096 buckets) + 8 bytes
    # per group, at most npoints / 8 + 2 groups
    npts = 262144
    extra = _ws(lib, 2000, 2, 5, 128, npoints=npts)[1] - b
    assert 32768 + 8 * (npts // 8 + 2) <= extra <= 32768 + 8 * (npts // 8 + 2) + 256


@pytest.mark.parametrize("n,kl,ku,P,npts", [(0, 0, 0, 32, 0), (5, 5, 0, 32, 0), (5, 0, 5, 32, 0), (5, -1, 0, 32, 0),
                                            (5, 1, 1, 0, 0), (5, 1, 1, 32, -1)])
def test_workspace_bytes_rejects(lib, n, kl, ku, P, npts):
    assert _ws(lib, n, kl, ku, P, npoints=npts)[0] == _native.PSA_EINVAL


def _call(lib, *, n=10, kl=1, ku=1, bands=1 << 20, grid=(-1.0, 1.0, -1.0, 1.0, 4, 4), eps=(0.1,),
          n_eps=None, idx=None, n_idx=0, sigma=1 << 21, opts=None, ws=1 << 22, ws_bytes=1 << 30):
    A = _native.PsaBand(n, kl, ku, bands)
    g = _native.PsaGrid(*grid)
    e = (ctypes.c_double * max(len(eps), 1))(*eps)
    o = opts if opts is not None else _native.PsaLanczosOpts(2, 100, 1e-13, 0)
    return lib.psa_sigma_min(ctypes.byref(A), ctypes.byref(g), e, len(eps) if n_eps is None else n_eps,
                             idx, n_idx, sigma, None, None, None, ctypes.byref(o), ws, ws_bytes, None)


@pytest.mark.parametrize("kw,code", [
    (dict(n=0), _native.PSA_EINVAL),
    (dict(kl=10), _native.PSA_EINVAL),
    (dict(bands=None), _native.PSA_EINVAL),
    (dict(sigma=None), _native.PSA_EINVAL),
    (dict(grid=(1.0, -1.0, -1.0, 1.0, 4, 4)), _native.PSA_EINVAL),
    (dict(grid=(-1.0, 1.0, -1.0, 1.0, 0, 4)), _native.PSA_EINVAL),
    (dict(grid=(-1.0, float("nan"), -1.0, 1.0, 4, 4)), _native.PSA_EINVAL),
    (dict(grid=(-1.0, 1.0, -1.0, 1.0, 65536, 65536)), _native.PSA_EINVAL),
    (dict(eps=(0.0,)), _native.PSA_EINVAL),
    (dict(eps=(-1e-3,)), _native.PSA_EINVAL),
    (dict(eps=(float("inf"),)), _native.PSA_EINVAL),
    (dict(n_eps=33), _native.PSA_EINVAL),
    (dict(n_idx=5, idx=None), _native.PSA_EINVAL),
    (dict(n_idx=-1), _native.PSA_EINVAL),
    (dict(opts=_native.PsaLanczosOpts(5, 4, 1e-13, 0)), _native.PSA_EINVAL),
    (dict(opts=_native.PsaLanczosOpts(2, 0, 1e-13, 0)), _native.PSA_EINVAL),
    (dict(opts=_native.PsaLanczosOpts(2, 70000, 1e-13, 0)), _native.PSA_EINVAL),
    (dict(opts=_native.PsaLanczosOpts(2, 10, -1.0, 0)), _native.PSA_EINVAL),
    (dict(n=20, kl=5, ku=1), _native.PSA_EUNSUPPORTED),
    (dict(n=20, kl=1, ku=9), _native.PSA_EUNSUPPORTED),
    (dict(n=400000, kl=2, ku=5), _native.PSA_EUNSUPPORTED),
    (dict(ws=None), _native.PSA_EWORKSPACE),
    (dict(ws=(1 << 22) + 8), _native.PSA_EWORKSPACE),
    (dict(ws_bytes=1000), _native.PSA_EWORKSPACE),
])
def test_sigma_min_rejects_bad_arguments(lib, kw, code):
    # every rejection happens on the host, before any device call
    assert _call(lib, **kw) == code


def _call_static(lib, *, n=10, kl=1, ku=1, bands=1 << 20, grid=(-1.0, 1.0, -1.0, 1.0, 4, 4), eps=(0.1,),
                 sigma=1 << 21, opts=None, null_grid=False):
    A = _native.PsaBand(n, kl, ku, bands)
    g = _native.PsaGrid(*grid)
    e = (ctypes.c_double * max(len(eps), 1))(*eps)
    o = opts if opts is not None else _native.PsaLanczosOpts(2, 1000, 1e-13, 0)
    return lib.psa_sigma_min_static(ctypes.byref(A), None if null_grid else ctypes.byref(g), e, len(eps),
                                    None, 0, sigma, None, None, None, ctypes.byref(o), None)


@pytest.mark.parametrize("kw,code", [
    # argument errors keep psa_sigma_min's codes even for problems beyond the static scratch
    (dict(n=20000, kl=5, ku=6), _native.PSA_EUNSUPPORTED),
    (dict(n=20000, kl=3, ku=9), _native.PSA_EUNSUPPORTED),
    (dict(n=20000, kl=3, ku=6, null_grid=True), _native.PSA_EINVAL),
    (dict(n=20000, kl=3, ku=6, eps=(0.0,)), _native.PSA_EINVAL),
    (dict(n=20000, kl=3, ku=6, sigma=None), _native.PSA_EINVAL),
    (dict(n=20000, kl=3, ku=6, bands=None), _native.PSA_EINVAL),
    # a valid problem that needs more than the scratch (about 134 MB for one warp)
    (dict(n=20000, kl=3, ku=6), _native.PSA_ESTATIC),
])
def test_static_entry_point_rejects_on_the_host(lib, kw, code):
    # every rejection happens before any device call (no GPU here)
    assert _call_static(lib, **kw) == code


@pytest.mark.parametrize("m,closed,null", [(0, 0, None), (-3, 1, None), (5, 2, None), (5, -1, None),
                                           (5, 0, "set"), (5, 1, "global"), (5, 0, "x")])
def test_point_features_over_a_set_rejects_on_the_host(lib, m, closed, null):
    g = _native.PsaGrid(-1.0, 1.0, -1.0, 1.0, 4, 4)
    p = {"set": 1 << 20, "global": 1 << 21, "x": 1 << 22}
    if null:
        p[null] = None
    rc = lib.psa_point_features_set(ctypes.byref(g), None, 0, 1 << 23, p["set"], m, closed, p["global"], p["x"], None)
    assert rc == _native.PSA_EINVAL


def test_point_set_stats_rejects_on_the_host(lib):
    assert lib.psa_point_set_stats(1 << 20, 0, 1 << 21, None) == _native.PSA_EINVAL
    assert lib.psa_point_set_stats(None, 4, 1 << 21, None) == _native.PSA_EINVAL
    assert lib.psa_point_set_stats(1 << 20, 4, None, None) == _native.PSA_EINVAL
