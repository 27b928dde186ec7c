"""psa_sigma_min_static, the entry point for callers that cannot allocate device memory.

Callers inside a host that hands out GPU memory once, a latency-bound loop or a
sandbox without allocator rights cannot provide the workspace that psa_sigma_min
takes. psa_sigma_min_static uses a fixed 64 MiB device array inside the library
instead. These checks call it through the C ABI, twice in a row (the array keeps
the previous call's contents), and compare sigma, masks, statuses and step counts
bitwise with psa_sigma_min on the same problem: a point's arithmetic does not
depend on how many points are in flight. One case has many groups per warp, so
that the work-order estimate pass and its schedule arrays in the shared array run
(and must be cleared) on both calls. The file is named to be collected last, and
it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2605_04550_gb300 as psa
from paper_2605_04550_gb300 import _native, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _static_call(lib, bands_t, kl, ku, grid, eps, opts):
    n = bands_t.shape[1]
    ny, nx = grid.ny, grid.nx
    sigma = torch.full((ny, nx), -1.0, dtype=torch.float64, device=DEV)
    mask = torch.zeros((ny, nx), dtype=torch.int32, device=DEV)
    status = torch.full((ny, nx), -1, dtype=torch.int8, device=DEV)
    steps = torch.zeros((ny, nx), dtype=torch.int32, device=DEV)
    A = _native.PsaBand(n, kl, ku, bands_t.data_ptr())
    g = _native.PsaGrid(grid.re_min, grid.re_max, grid.im_min, grid.im_max, nx, ny)
    e = (ctypes.c_double * len(eps))(*eps)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.psa_sigma_min_static(ctypes.byref(A), ctypes.byref(g), e, len(eps), None, 0,
                                  sigma.data_ptr(), mask.data_ptr(), status.data_ptr(), steps.data_ptr(),
                                  ctypes.byref(opts._c()), stream)
    torch.cuda.synchronize()
    return (rc, sigma.cpu().numpy().ravel(), mask.cpu().numpy().view(np.uint32).ravel(),
            status.cpu().numpy().ravel(), steps.cpu().numpy().ravel())


@pytest.mark.parametrize("case", ["grcar", "toeplitz", "toeplitz_ordered"])
def test_static_scratch_matches_workspace_entry_point_twice(case):
    lib = _native.load()
    if case == "grcar":
        bands, kl, ku = inputs.grcar(100)
        grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 64, 48)
    elif case == "toeplitz":
        bands, kl, ku, a = inputs.random_toeplitz(600, 2, 5, seed=0)
        grid = inputs.toeplitz_symbol_grid(a, kl, ku, 40, 33)
    else:
        # 512 groups of 32 points for the 13 warps that fit in the array: the estimate
        # pass, the bucket histogram and the work order live in the array too
        bands, kl, ku, a = inputs.random_toeplitz(600, 2, 5, seed=1)
        grid = inputs.toeplitz_symbol_grid(a, kl, ku, 128, 128)
    eps = inputs.EPS_LEVELS_8
    opts = psa.LanczosOpts()
    b = torch.as_tensor(bands, device=DEV)
    ref = psa.sigma_min(b, kl, ku, grid, eps=eps, opts=opts)
    torch.cuda.synchronize()
    ref_s = ref.sigma.cpu().numpy().ravel()
    ref_m = ref.mask.cpu().numpy().view(np.uint32).ravel()
    ref_st = ref.status.cpu().numpy().ravel()
    ref_k = ref.steps.cpu().numpy().ravel()
    for call in range(2):
        rc, s, m, st, k = _static_call(lib, b, kl, ku, grid, eps, opts)
        assert rc == _native.PSA_OK, (call, rc)
        np.testing.assert_array_equal(s, ref_s)
        np.testing.assert_array_equal(k, ref_k)
        np.testing.assert_array_equal(m, ref_m)
        np.testing.assert_array_equal(st, ref_st)


def test_static_scratch_rejects_problems_beyond_its_size():
    lib = _native.load()
    # n = 20000 with 1000 Lanczos steps needs ~134 MB for 32 points in flight
    b = torch.zeros((3 + 6 + 1, 20000), dtype=torch.complex128, device=DEV)
    grid = inputs.Grid(-1.0, 1.0, -1.0, 1.0, 4, 4)
    rc, s, _, _, _ = _static_call(lib, b, 3, 6, grid, (0.1,), psa.LanczosOpts())
    assert rc == _native.PSA_ESTATIC
    assert np.all(s == -1.0)          # nothing was launched
    assert b"static scratch" in lib.psa_strerror(rc)
