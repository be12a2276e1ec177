"""ov_apply_HW_noalloc against ov_apply_HW, through the C ABI (GPU).

The allocation-free entry point exists for callers that cannot call cudaMalloc
(a code that gives all of HBM to its own pool, a framework allocator that must not
be bypassed, work enqueued during graph capture).  Its scratch is one fixed device
array shared by every call, so two calls in a row must each give the result of the
ordinary entry point: nothing may leak from the previous call.  This file is
collected last so that a failure here cannot stop the other tests from running.
"""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import M0, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_noalloc_matches_apply_HW_on_two_calls(gpu_lib):
    import torch

    dims = (8, 8, 8, 8)
    U = S.su3_links(dims, 0.5, 4001)
    Ud = to_dev(U)
    ctx = gpu_lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(Ud)
    for call, seed in enumerate((4002, 4003)):
        nrhs = 2 + call
        psi = to_dev(S.gaussian_spinor(dims, seed, n=nrhs))
        want = torch.empty_like(psi)
        ctx.apply_HW(psi, want, nrhs, gpu_lib.OV_FP64)
        got = torch.full_like(psi, float("nan"))
        rc = gpu_lib.apply_HW_noalloc(dims, -1, M0, Ud, psi, got, nrhs)
        assert rc == gpu_lib.OV_OK
        torch.cuda.synchronize()
        w, g = to_host(want), to_host(got)
        assert np.abs(g - w).max() <= 1e-14 * np.abs(w).max(), f"call {call}"
    ctx.close()


def test_noalloc_rejects_requests_beyond_its_scratch(gpu_lib):
    import torch

    dims = (16, 16, 16, 16)  # gauge staging alone is 37.7 MB > 16 MiB
    Ud = torch.zeros((4, 16, 16, 16, 16, 3, 3), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((16, 16, 16, 16, 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    assert gpu_lib.apply_HW_noalloc(dims, -1, M0, Ud, psi, out, 1) == gpu_lib.OV_ERR_SCRATCH_TOO_SMALL
    small = (4, 4, 4, 4)
    x = torch.zeros((2, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    assert gpu_lib.apply_HW_noalloc(small, -1, M0, Ud, x[0], x[0], 1) == gpu_lib.OV_ERR_INVALID_ARG
