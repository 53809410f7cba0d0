"""Failure paths on the GPU that fault, trap and hang nothing: an allocation the device
cannot satisfy reports RC_ERR_OOM, and the library's bounded device-side wait gives up on an
mbarrier nobody completes and reports RC_ERR_TIMEOUT; afterwards the context still runs a
formal solution that matches the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2408_14425_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rcx():
    from paper_2408_14425_b300 import build, rcx
    build.build()
    return rcx


def test_out_of_memory_is_reported():
    rcx = _rcx()
    L = rcx.load()
    p = rcx.Plan(8192, 8192, 3)
    # 8192^2 cells x 2^20 wavelengths of packed field is petabytes
    assert L.rc_plan_reserve(p.handle, 1 << 20) == -2
    assert b"scratch allocation failed" in L.rc_last_error()
    assert torch.cuda.mem_get_info()[0] > 0          # nothing was left allocated by the failure


def test_bounded_wait_times_out_and_context_survives():
    rcx = _rcx()
    L = rcx.load()
    assert L.rc_selftest_bounded_wait(None) == -4     # RC_ERR_TIMEOUT, as designed
    assert b"gave up" in L.rc_last_error()
    chi, eta = W.disc_field()                        # [1][64][64]
    J = rcx.Plan(64, 64, 5).formal_solve(torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda())
    J_ref, _, _ = oracle.rc_solve(chi.astype(np.float64), eta.astype(np.float64), 5)
    J = J.cpu().numpy()
    assert np.all(np.abs(J - J_ref) <= 1e-3 * np.abs(J_ref) + 1e-7 * np.abs(J_ref).max())
