"""Host-side checks of the batch calls of the C ABI (no GPU needed): the plan groups
the matrices by band shape, orders each class by decreasing n and lays out tiles,
start vectors and outputs as documented; the workspace is sized from the plan; bad
entries and arguments are rejected before any device call."""
import ctypes

import numpy as np
import pytest

from paper_2605_04550_gb300 import _native
from paper_2605_04550_gb300.build import build_library

MAX_CLASSES = 5 * 9
CLASS_OFF = 256
CLASS_BYTES, MAT_BYTES = 40, 88
MAT_OFF = CLASS_OFF + ((MAX_CLASSES * CLASS_BYTES + 255) // 256) * 256


class PlanHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_int32), ("nmat", ctypes.c_int32), ("nclass", ctypes.c_int32),
                ("max_n", ctypes.c_int32), ("q1_total", ctypes.c_int64), ("max_ngroups", ctypes.c_int64)]


class PlanClass(ctypes.Structure):
    _fields_ = [("kl", ctypes.c_int32), ("ku", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("first", ctypes.c_int32), ("count", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("ngroups", ctypes.c_int64), ("nchunks", ctypes.c_int64)]


class PlanMat(ctypes.Structure):
    _fields_ = [("bands", ctypes.c_void_p), ("n", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("pad", ctypes.c_int32), ("re_min", ctypes.c_double),
                ("im_min", ctypes.c_double), ("hx", ctypes.c_double), ("hy", ctypes.c_double),
                ("out_off", ctypes.c_int64), ("gstart", ctypes.c_int64), ("q1_off", ctypes.c_int64),
                ("estart", ctypes.c_int64)]


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _native.load()


def _entries(specs):
    """specs: (n, kl, ku, nx, ny) per matrix; outputs laid out consecutively."""
    E = (_native.PsaBatchEntry * len(specs))()
    off = 0
    for m, (n, kl, ku, nx, ny) in enumerate(specs):
        E[m].A = _native.PsaBand(n, kl, ku, 0x1000 * (m + 1))  # never dereferenced on the host
        E[m].g = _native.PsaGrid(-1.0 - m, 1.0 + m, -2.0, 2.0, nx, ny)
        E[m].out_offset = off
        off += nx * ny
    return E


def _plan(lib, specs):
    E = _entries(specs)
    nb = ctypes.c_size_t()
    assert lib.psa_batch_plan_bytes(len(specs), ctypes.byref(nb)) == 0
    buf = ctypes.create_string_buffer(nb.value)
    rc = lib.psa_batch_plan(E, len(specs), buf, nb.value)
    return rc, buf, E


def _parse(buf):
    H = PlanHeader.from_buffer_copy(buf.raw[:ctypes.sizeof(PlanHeader)])
    C = [PlanClass.from_buffer_copy(buf.raw[CLASS_OFF + CLASS_BYTES * c:CLASS_OFF + CLASS_BYTES * (c + 1)])
         for c in range(H.nclass)]
    sz = ctypes.sizeof(PlanMat)
    M = [PlanMat.from_buffer_copy(buf.raw[MAT_OFF + sz * m:MAT_OFF + sz * (m + 1)]) for m in range(H.nmat)]
    return H, C, M


def test_plan_struct_sizes_match_the_library(lib):
    assert ctypes.sizeof(PlanClass) == CLASS_BYTES and ctypes.sizeof(PlanMat) == MAT_BYTES
    nb = ctypes.c_size_t()
    assert lib.psa_batch_plan_bytes(10, ctypes.byref(nb)) == 0
    assert nb.value == MAT_OFF + -(-10 * MAT_BYTES // 256) * 256


def test_plan_groups_classes_and_orders_by_decreasing_n(lib):
    rng = np.random.default_rng(0)
    specs = [(int(rng.integers(10, 3000)), int(rng.integers(0, 5)), int(rng.integers(0, 9)),
              int(rng.integers(1, 40)), int(rng.integers(1, 40))) for _ in range(60)]
    specs = [(max(n, kl + 1, ku + 1), kl, ku, nx, ny) for n, kl, ku, nx, ny in specs]
    rc, buf, E = _plan(lib, specs)
    assert rc == 0
    H, C, M = _parse(buf)
    assert H.magic == 0x50534142 and H.nmat == 60
    shapes = sorted({(kl, ku) for _, kl, ku, _, _ in specs})
    assert [(c.kl, c.ku) for c in C] == shapes
    assert H.nclass == len(shapes)
    seen = set()
    q1 = 0
    for c in C:
        members = M[c.first:c.first + c.count]
        # every matrix of the class, largest first
        assert sorted(m.n for m in members)[::-1] == [m.n for m in members]
        assert c.n_max == members[0].n
        g = ch = 0
        for m in members:
            src = (m.bands // 0x1000) - 1
            seen.add(src)
            n, kl, ku, nx, ny = specs[src]
            assert (m.n, m.nx, m.ny, kl, ku) == (n, nx, ny, c.kl, c.ku)
            assert m.out_off == E[src].out_offset
            assert m.gstart == g and m.estart == ch
            assert m.q1_off == q1
            tiles = ((nx + 7) // 8) * ((ny + 3) // 4)
            g += tiles
            ch += (tiles + 31) // 32
            q1 += n
            assert m.hx == pytest.approx(2 * (1.0 + src) / (nx - 1) if nx > 1 else 0.0)
            assert m.re_min == -1.0 - src
        assert (c.ngroups, c.nchunks) == (g, ch)
    assert seen == set(range(60))
    assert H.q1_total == q1 == sum(s[0] for s in specs)
    assert H.max_ngroups == max(c.ngroups for c in C)
    assert H.max_n == max(s[0] for s in specs)


@pytest.mark.parametrize("spec,code", [
    ((10, 5, 1, 4, 4), _native.PSA_EUNSUPPORTED),
    ((10, 1, 9, 4, 4), _native.PSA_EUNSUPPORTED),
    ((0, 0, 0, 4, 4), _native.PSA_EINVAL),
    ((3, 3, 0, 4, 4), _native.PSA_EINVAL),
    ((10, 1, 1, 0, 4), _native.PSA_EINVAL),
    ((10, 1, 1, 65536, 65536), _native.PSA_EINVAL),
])
def test_plan_rejects_bad_entries(lib, spec, code):
    assert _plan(lib, [(50, 1, 1, 8, 8), spec])[0] == code


def test_plan_rejects_null_bands_negative_offset_and_small_buffer(lib):
    E = _entries([(50, 1, 1, 8, 8), (60, 2, 2, 8, 8)])
    nb = ctypes.c_size_t()
    lib.psa_batch_plan_bytes(2, ctypes.byref(nb))
    buf = ctypes.create_string_buffer(nb.value)
    assert lib.psa_batch_plan(E, 2, buf, nb.value - 1) == _native.PSA_EINVAL
    assert lib.psa_batch_plan(E, 2, None, nb.value) == _native.PSA_EINVAL
    assert lib.psa_batch_plan(E, -1, buf, nb.value) == _native.PSA_EINVAL
    E[1].out_offset = -1
    assert lib.psa_batch_plan(E, 2, buf, nb.value) == _native.PSA_EINVAL
    E[1].out_offset = 64
    E[1].A.bands = None
    assert lib.psa_batch_plan(E, 2, buf, nb.value) == _native.PSA_EINVAL
    assert lib.psa_batch_plan_bytes(-1, ctypes.byref(nb)) == _native.PSA_EINVAL


def _align(x):
    return -(-x // 256) * 256


def test_batch_workspace_bytes_layout(lib):
    specs = [(2000, 2, 5, 128, 128), (800, 2, 5, 128, 128), (3000, 1, 3, 64, 64), (100, 4, 8, 16, 16)]
    rc, buf, _ = _plan(lib, specs)
    assert rc == 0
    H, C, _ = _parse(buf)
    kmax = 1000
    o = _native.PsaLanczosOpts(2, kmax, 1e-13, 0)
    pif = 4096
    out = ctypes.c_size_t()
    warp = []
    for c in C:
        row = (2 * c.kl + c.ku + 1 + 3) * 512 + 128
        wb = _align(c.n_max * row + 2 * kmax * 32 * 8)
        warp.append(min(pif // 32, c.ngroups) * wb)
    for streams in (1, 2, 8):
        assert lib.psa_batch_workspace_bytes(buf, ctypes.byref(o), pif, streams, ctypes.byref(out)) == 0
        # counters, matrix flags, start vectors; per stream a schedule and a region
        fixed = _align(4 * 2 * MAX_CLASSES) + _align(4 * 4) + _align(16 * sum(s[0] for s in specs))
        sched = _align(4 * (2 * 4096 + 2 * H.max_ngroups))
        assert out.value == fixed + streams * (sched + max(warp))
    for bad in ((buf, 0, 1), (None, 32, 1), (buf, 32, 0), (buf, 32, 9)):
        assert lib.psa_batch_workspace_bytes(bad[0], ctypes.byref(o), bad[1], bad[2],
                                             ctypes.byref(out)) == _native.PSA_EINVAL


def test_sigma_min_batched_rejects_on_the_host(lib):
    rc, buf, _ = _plan(lib, [(50, 1, 1, 8, 8)])
    assert rc == 0
    o = _native.PsaLanczosOpts(2, 100, 1e-13, 0)
    eps = (ctypes.c_double * 1)(0.1)

    def call(plan=buf, dev=1 << 20, e=eps, ne=1, sigma=1 << 21, pif=0, order=0, ws=1 << 22, wsb=1 << 30,
             stream=None, aux=(), n_aux=None):
        arr = (ctypes.c_void_p * max(len(aux), 1))(*aux)
        return lib.psa_sigma_min_batched(plan, dev, e, ne, sigma, None, None, None, ctypes.byref(o), pif, order,
                                         ws, wsb, stream, arr, len(aux) if n_aux is None else n_aux)
    bad = ctypes.create_string_buffer(len(buf.raw))
    assert call(plan=bad) == _native.PSA_EINVAL            # header does not check
    assert call(dev=None) == _native.PSA_EINVAL
    assert call(dev=(1 << 20) + 16) == _native.PSA_EINVAL  # plan copy not 256-byte aligned
    assert call(sigma=None) == _native.PSA_EINVAL
    assert call(ne=33) == _native.PSA_EINVAL
    assert call(e=(ctypes.c_double * 1)(0.0)) == _native.PSA_EINVAL
    assert call(order=3) == _native.PSA_EINVAL
    assert call(pif=-1) == _native.PSA_EINVAL
    assert call(ws=None) == _native.PSA_EWORKSPACE
    assert call(wsb=1024) == _native.PSA_EWORKSPACE
    # auxiliary streams: other streams than the call's, all different, at most 7
    assert call(stream=0x1234, aux=(0x1234,)) == _native.PSA_EINVAL
    assert call(stream=0x1234, aux=(0x10, 0x20, 0x10)) == _native.PSA_EINVAL
    assert call(stream=0x1234, aux=tuple(range(0x10, 0x18))) == _native.PSA_EINVAL
    assert call(n_aux=-1) == _native.PSA_EINVAL
