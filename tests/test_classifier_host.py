"""Host-side checks of the classifier and feature entry points of the C ABI (no GPU):
workspace sizes as documented and every argument rejection taken before any device
call; the empty batch is a no-op."""
import ctypes

import pytest

from paper_2605_04550_gb300 import _native
from paper_2605_04550_gb300.build import build_library

IN, HID, P = _native.MLP_IN, _native.MLP_HIDDEN, _native.MLP_PARAMS


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _native.load()


def _align(x):
    return -(-x // 256) * 256


def test_parameter_count_matches_the_layout():
    assert P == HID * IN + HID + 2 * (HID * HID + HID) + HID + 1


def test_mlp_workspace_bytes(lib):
    out = ctypes.c_size_t()
    # forward: BF16 weights (3 matrices) + three BF16 activation buffers of the pass's rows
    assert lib.psa_mlp_workspace_bytes(1000, 0, ctypes.byref(out)) == 0
    rows = 1024  # rounded up to the 128-row tile
    expect = _align(2 * HID * IN) + 2 * _align(2 * HID * HID) + 3 * _align(2 * HID * rows)
    assert out.value == expect
    # passes of at most 131072 rows
    lib.psa_mlp_workspace_bytes(10 ** 7, 0, ctypes.byref(out))
    big = out.value
    lib.psa_mlp_workspace_bytes(131072, 0, ctypes.byref(out))
    assert big == out.value
    # training adds transposed weights, transposed activations, pre-activations, gradients
    assert lib.psa_mlp_workspace_bytes(512, 1, ctypes.byref(out)) == 0
    assert out.value > expect
    assert lib.psa_mlp_workspace_bytes(-1, 0, ctypes.byref(out)) == _native.PSA_EINVAL
    assert lib.psa_mlp_workspace_bytes(10, 0, None) == _native.PSA_EINVAL


def test_gemm_rejects(lib):
    A, B, C = 1 << 20, 1 << 21, 1 << 22

    def g(a=A, lda=128, b=B, ldb=128, M=256, N=256, K=128, c=C, ldc=256):
        return lib.psa_gemm_bf16(a, lda, b, ldb, M, N, K, c, ldc, None)
    assert g(N=200) == _native.PSA_EINVAL          # N not a multiple of 128
    assert g(K=100, lda=128, ldb=128) == _native.PSA_EINVAL  # K not a multiple of 64
    assert g(lda=64) == _native.PSA_EINVAL         # lda < K
    assert g(ldc=128) == _native.PSA_EINVAL        # ldc < N
    assert g(lda=132, K=128) == _native.PSA_EINVAL  # lda not a multiple of 8
    assert g(a=A + 8) == _native.PSA_EINVAL        # not 16-byte aligned
    assert g(a=None) == _native.PSA_EINVAL
    assert g(M=-1) == _native.PSA_EINVAL
    assert g(M=0) == _native.PSA_OK                # nothing to do, nothing launched


def test_mlp_forward_and_train_reject(lib):
    th, x, y, pr, ws = 1 << 20, 1 << 24, 1 << 25, 1 << 26, 1 << 28
    assert lib.psa_mlp_forward(None, x, 10, pr, ws, 1 << 30, None) == _native.PSA_EINVAL
    assert lib.psa_mlp_forward(th, x + 8, 10, pr, ws, 1 << 30, None) == _native.PSA_EINVAL
    assert lib.psa_mlp_forward(th, x, 10, pr, ws, 10, None) == _native.PSA_EWORKSPACE
    assert lib.psa_mlp_forward(th, x, 10, pr, ws + 16, 1 << 30, None) == _native.PSA_EWORKSPACE
    assert lib.psa_mlp_forward(th, x, 0, pr, ws, 1 << 30, None) == _native.PSA_OK

    def t(rows=512, step=1, lr=1e-3, wsb=1 << 30, w=ws):
        return lib.psa_mlp_train_step(th, 1 << 27, 1 << 29, step, lr, x, y, rows, 1 << 30, w, wsb, None)
    assert t(rows=500) == _native.PSA_EINVAL        # not a multiple of 128
    assert t(rows=0) == _native.PSA_EINVAL
    assert t(step=0) == _native.PSA_EINVAL
    assert t(lr=0.0) == _native.PSA_EINVAL
    assert t(wsb=1024) == _native.PSA_EWORKSPACE


def test_feature_entry_points_reject(lib):
    A = _native.PsaBand(100, 1, 3, 1 << 20)
    st, sym, glob, x = 1 << 21, 1 << 22, 1 << 23, 1 << 24
    assert lib.psa_matrix_stats(None, st, sym, None) == _native.PSA_EINVAL
    assert lib.psa_matrix_stats(ctypes.byref(_native.PsaBand(100, 5, 8, 1 << 20)), st, sym, None) == \
        _native.PSA_EUNSUPPORTED                     # 14 bands > 13
    assert lib.psa_matrix_stats(ctypes.byref(_native.PsaBand(3, 4, 0, 1 << 20)), st, sym, None) == _native.PSA_EINVAL
    assert lib.psa_matrix_stats(ctypes.byref(A), None, sym, None) == _native.PSA_EINVAL
    assert lib.psa_global_features(st, None, 0.01, glob, None) == _native.PSA_EINVAL
    assert lib.psa_global_features(st, sym, 0.0, glob, None) == _native.PSA_EINVAL
    assert lib.psa_global_features(st, sym, float("nan"), glob, None) == _native.PSA_EINVAL
    g = _native.PsaGrid(-1.0, 1.0, -1.0, 1.0, 10, 10)
    bad = _native.PsaGrid(1.0, -1.0, -1.0, 1.0, 10, 10)
    assert lib.psa_point_features(ctypes.byref(bad), None, 0, st, sym, glob, x, None) == _native.PSA_EINVAL
    assert lib.psa_point_features(ctypes.byref(g), None, 5, st, sym, glob, x, None) == _native.PSA_EINVAL
    assert lib.psa_point_features(ctypes.byref(g), None, 0, st, sym, glob, x + 2, None) == _native.PSA_EINVAL
    assert lib.psa_point_features(ctypes.byref(g), 1 << 25, 0, st, sym, glob, x, None) == _native.PSA_OK  # empty list
    assert lib.psa_region(None, 0.5, 10, 10, 2, x, None) == _native.PSA_EINVAL
    assert lib.psa_region(st, 0.5, 0, 10, 2, x, None) == _native.PSA_EINVAL
    assert lib.psa_region(st, 0.5, 10, 10, 65, x, None) == _native.PSA_EINVAL
    assert lib.psa_tile_slots(None, 10, 10, x, None) == _native.PSA_EINVAL
    assert lib.psa_tile_slots(st, 10, -1, x, None) == _native.PSA_EINVAL


def test_empty_batch_is_a_no_op(lib):
    nb = ctypes.c_size_t()
    assert lib.psa_batch_plan_bytes(0, ctypes.byref(nb)) == 0
    buf = ctypes.create_string_buffer(nb.value)
    assert lib.psa_batch_plan(None, 0, buf, nb.value) == 0
    o = _native.PsaLanczosOpts(2, 100, 1e-13, 0)
    out = ctypes.c_size_t()
    assert lib.psa_batch_workspace_bytes(buf, ctypes.byref(o), 32, 1, ctypes.byref(out)) == 0
    arr = (ctypes.c_void_p * 1)()
    # nothing to evaluate: returns before any device call
    assert lib.psa_sigma_min_batched(buf, 1 << 20, None, 0, 1 << 21, None, None, None, ctypes.byref(o), 0, 0,
                                     1 << 22, out.value, None, arr, 0) == 0
