"""ov_apply_HW_noalloc against the oracle and against ov_apply_HW, through the C ABI (GPU).

The allocation-free entry point exists for callers that cannot call cudaMalloc (a
code that gives all of HBM to its own pool, a framework allocator that must not be
bypassed).  Its scratch is one fixed device array shared by every call, so two calls
in a row must each give the right result: nothing may leak from the previous call.
This file is collected last so that a failure here cannot stop the other tests from
running.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from oracle import cimpl
from tests.gpu_common import M0, to_dev, to_host

pytestmark = pytest.mark.gpu


def _elem_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (3, 5, 4, 6)], ids=["8^4", "3x5x4x6"])
@pytest.mark.parametrize("bc_t", [-1, 1])
def test_noalloc_matches_oracle_on_two_calls(gpu_lib, dims, bc_t):
    """Element by element against the C oracle's H_W (Eq. 1), periodic and antiperiodic
    time, cubic and ragged lattices, two calls in a row with different source counts."""
    import torch

    U = S.su3_links(dims, 0.5, 4001)
    Ud = to_dev(U)
    for call, seed in enumerate((4002, 4003)):
        nrhs = 2 + call
        psi = S.gaussian_spinor(dims, seed, n=nrhs)
        got = torch.full_like(to_dev(psi), float("nan"))
        rc = gpu_lib.apply_HW_noalloc(dims, bc_t, M0, Ud, to_dev(psi), got, nrhs)
        assert rc == gpu_lib.OV_OK
        torch.cuda.synchronize()
        g = to_host(got)
        for k in range(nrhs):
            want = cimpl.hw_apply(U, psi[k], M0, bc_t=bc_t)
            assert _elem_err(g[k], want) <= 1e-14, (call, k)


def test_noalloc_matches_apply_HW_on_two_calls(gpu_lib):
    """The same as the context-based entry point, on a non-cubic lattice with several
    right-hand sides, twice in a row."""
    import torch

    dims = (6, 4, 8, 10)
    U = S.su3_links(dims, 0.5, 4011)
    Ud = to_dev(U)
    ctx = gpu_lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(Ud)
    for call, seed in enumerate((4012, 4013)):
        nrhs = 5 - 2 * call
        psi = to_dev(S.gaussian_spinor(dims, seed, n=nrhs))
        want = torch.empty_like(psi)
        ctx.apply_HW(psi, want, nrhs, gpu_lib.OV_FP64)
        got = torch.full_like(psi, float("nan"))
        assert gpu_lib.apply_HW_noalloc(dims, -1, M0, Ud, psi, got, nrhs) == gpu_lib.OV_OK
        torch.cuda.synchronize()
        assert _elem_err(to_host(got), to_host(want)) <= 1e-14, call
    ctx.close()


def test_noalloc_rejects_bad_requests(gpu_lib):
    import torch

    dims = (16, 16, 16, 16)  # gauge staging alone is 37.7 MB > 16 MiB
    Ud = torch.zeros((4, 16, 16, 16, 16, 3, 3), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((16, 16, 16, 16, 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    assert gpu_lib.apply_HW_noalloc(dims, -1, M0, Ud, psi, out, 1) == gpu_lib.OV_ERR_SCRATCH_TOO_SMALL
    # extents whose product overflows 64 bits: rejected by size, nothing launched
    huge = (1 << 30, 1 << 30, 1 << 30, 1 << 30)
    assert gpu_lib.apply_HW_noalloc(huge, -1, M0, Ud, psi, out, 1) == gpu_lib.OV_ERR_SCRATCH_TOO_SMALL
    # too many right-hand sides for the scratch on a small lattice
    small = (4, 4, 4, 4)
    x = torch.zeros((2, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    assert gpu_lib.apply_HW_noalloc(small, -1, M0, Ud, x[0], x[1], 100000) == gpu_lib.OV_ERR_SCRATCH_TOO_SMALL
    assert gpu_lib.apply_HW_noalloc(small, -1, M0, Ud, x[0], x[0], 1) == gpu_lib.OV_ERR_INVALID_ARG
    assert gpu_lib.apply_HW_noalloc(small, 0, M0, Ud, x[0], x[1], 1) == gpu_lib.OV_ERR_INVALID_ARG
    assert gpu_lib.apply_HW_noalloc(small, -1, float("nan"), Ud, x[0], x[1], 1) == gpu_lib.OV_ERR_INVALID_ARG
    assert gpu_lib.apply_HW_noalloc(small, -1, float("inf"), Ud, x[0], x[1], 1) == gpu_lib.OV_ERR_INVALID_ARG


def test_noalloc_leaves_a_pending_caller_error_alone(gpu_lib):
    """A (harmless) error the caller's own earlier CUDA call left pending is neither
    cleared by the entry point nor reported as its failure."""
    import torch

    try:
        rt = ctypes.CDLL("libcudart.so.13")
    except OSError:
        pytest.skip("CUDA runtime not loadable by soname")
    rt.cudaPeekAtLastError.restype = ctypes.c_int
    rt.cudaGetLastError.restype = ctypes.c_int
    rt.cudaSetDevice.restype = ctypes.c_int
    torch.cuda.synchronize()
    rt.cudaGetLastError()
    dev = torch.cuda.current_device()
    bad = rt.cudaSetDevice(ctypes.c_int(10 ** 6))  # invalid ordinal: an error, nothing else
    assert bad != 0
    rt.cudaSetDevice(ctypes.c_int(dev))
    if rt.cudaPeekAtLastError() != bad:
        rt.cudaGetLastError()
        pytest.skip("this runtime does not keep the invalid-device error pending")
    dims = (4, 4, 4, 4)
    U = S.su3_links(dims, 0.5, 4021)
    psi = S.gaussian_spinor(dims, 4022)
    got = torch.empty_like(to_dev(psi))
    rc = gpu_lib.apply_HW_noalloc(dims, -1, M0, to_dev(U), to_dev(psi), got, 1)
    pending = rt.cudaPeekAtLastError()
    rt.cudaGetLastError()
    assert rc == gpu_lib.OV_OK
    assert pending == bad
    torch.cuda.synchronize()
    assert _elem_err(to_host(got), cimpl.hw_apply(U, psi, M0)) <= 1e-14
