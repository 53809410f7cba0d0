"""rc_formal_solve_noalloc: the formal solution for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc -- their device memory belongs to
another allocator or to a budget fixed at start-up.  This entry point keeps its scratch
in a static device array inside librcx.so.  The test calls it through the C ABI twice
in a row (different problems, so the second call runs on the first call's leftovers)
and checks each result against the allocating entry point rc_formal_solve, within the
parity tolerance of the other tests (1e-3 relative).  It lives in a file that pytest
collects last and passes both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    from paper_2408_14425_b300 import build, rcx
    build.build()
    return rcx


def _close(a, b, rtol=1e-3):
    a = a.double()
    b = b.double()
    floor = 1e-7 * b.abs().max()
    assert torch.isfinite(a).all()
    assert bool(((a - b).abs() <= rtol * b.abs() + floor).all()), \
        f"max rel diff {((a - b).abs() / b.abs().clamp_min(1e-30)).max().item():.3e}"


def _problem(seed, nl, nx, nz):
    rng = np.random.default_rng(seed)
    chi = (10 ** rng.uniform(-4, 1, size=(nl, nz, nx))).astype(np.float32)
    eta = (chi * 10 ** rng.uniform(-1, 1, size=chi.shape)).astype(np.float32)
    return torch.from_numpy(chi).cuda(), torch.from_numpy(eta).cuda()


def test_noalloc_matches_allocating_entry_point_twice():
    rcx = _lib()
    L = rcx.load()
    torch.cuda.init()
    cases = [(11, 5, 96, 80, 5, 4, 1.0), (12, 7, 128, 128, 6, 4, 1.5)]
    for seed, nl, nx, nz, C, W0, L0 in cases:
        chi, eta = _problem(seed, nl, nx, nz)
        J_na = torch.full_like(chi, float("nan"))
        alo_na = torch.full_like(chi, float("nan"))
        g = rcx.rc_grid(nx, nz, 1.0)
        st = L.rc_formal_solve_noalloc(ctypes.byref(g), C, W0, L0, ctypes.c_void_p(chi.data_ptr()),
                                       ctypes.c_void_p(eta.data_ptr()), nl,
                                       ctypes.c_void_p(J_na.data_ptr()),
                                       ctypes.c_void_p(alo_na.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, L.rc_last_error()
        plan = rcx.Plan(nx, nz, C, dirs0=W0, interval0=L0)
        J_ref, alo_ref = plan.formal_solve(chi, eta, want_alo=True)
        torch.cuda.synchronize()
        _close(J_na, J_ref)
        _close(alo_na, alo_ref)
        plan.close()


def test_noalloc_rejects_problems_beyond_its_static_scratch():
    rcx = _lib()
    L = rcx.load()
    chi = torch.ones((64, 512, 512), device="cuda")
    g = rcx.rc_grid(512, 512, 1.0)
    st = L.rc_formal_solve_noalloc(ctypes.byref(g), 7, 4, 1.0, ctypes.c_void_p(chi.data_ptr()),
                                   ctypes.c_void_p(chi.data_ptr()), 64,
                                   ctypes.c_void_p(chi.data_ptr()), None, None)
    assert st == -1
    assert b"static array" in L.rc_last_error()


def test_noalloc_calls_leave_device_free_memory_unchanged():
    """Once warm (module and kernels loaded by the first calls), further calls must not change
    the device's free memory: a buffer that a later change kept between calls (a cached scale
    or work list) would show up here."""
    rcx = _lib()
    L = rcx.load()
    chi, eta = _problem(21, 6, 112, 96)
    J = torch.empty_like(chi)
    g = rcx.rc_grid(112, 96, 1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        st = L.rc_formal_solve_noalloc(ctypes.byref(g), 6, 4, 1.0, ctypes.c_void_p(chi.data_ptr()),
                                       ctypes.c_void_p(eta.data_ptr()), 6,
                                       ctypes.c_void_p(J.data_ptr()), None, stream)
        assert st == 0, L.rc_last_error()

    for _ in range(2):
        call()
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
