"""af_step_noalloc: the FP64 step for callers that may not allocate device
memory (a fixed device-memory budget, or a host runtime that owns every
allocation).  It must give the same result as the regular handle-based step,
on two calls in a row (the second reusing the static work area the first one
left behind).  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_2605_12915_gb300 as af
from workloads import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def rel_linf(a, b):
    num = np.max(np.abs(a - b), axis=(1, 2))
    den = np.maximum(np.max(np.abs(b), axis=(1, 2)), 1e-300)
    return float(np.max(num / den))


def _lib():
    af._build.build()
    lib = af.load()
    fn = lib.af_step_noalloc
    fn.argtypes = [ctypes.POINTER(af.AfGrid), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                   ctypes.POINTER(af.AfState), ctypes.POINTER(af.AfState), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _state(t, n):
    return af._state_struct(t.data_ptr(), n)


@pytest.mark.parametrize("variant", [af.AF_TAI, af.AF_RB])
def test_noalloc_matches_handle_step_twice(variant):
    torch = pytest.importorskip("torch")
    step_noalloc = _lib()
    P = I.random_smooth(90, 70, seed=12, amp=0.06)
    n = P.grid.nx * P.grid.ny
    dt = P.dt * (0.6 if variant == af.AF_RB else 1.0)
    g = af.AfGrid(P.grid.nx, P.grid.ny, P.grid.h)

    # the regular entry points, two steps
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64",
                  variant="tai" if variant == af.AF_TAI else "rb")
    s.step(dt, 1)
    want1 = s.state()
    s.step(dt, 1)
    want2 = s.state()
    s.close()

    # the allocation-free entry point, two calls in a row on the same stream
    a = torch.from_numpy(P.state).cuda()
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    rc = step_noalloc(ctypes.byref(g), P.gamma, dt, variant, ctypes.byref(_state(a, n)),
                      ctypes.byref(_state(b, n)), ctypes.c_void_p(stream))
    assert rc == af.AF_OK
    rc = step_noalloc(ctypes.byref(g), P.gamma, dt, variant, ctypes.byref(_state(b, n)),
                      ctypes.byref(_state(c, n)), ctypes.c_void_p(stream))
    assert rc == af.AF_OK
    assert rel_linf(b.cpu().numpy(), want1) < TOL64
    assert rel_linf(c.cpu().numpy(), want2) < TOL64


def test_noalloc_rejects_grids_beyond_its_work_area():
    torch = pytest.importorskip("torch")
    step_noalloc = _lib()
    nx, ny = 130, 130  # 16900 cells > 128 * 128
    g = af.AfGrid(nx, ny, 0.01)
    a = torch.zeros((16, ny, nx), dtype=torch.float64, device="cuda")
    st = _state(a, nx * ny)
    rc = step_noalloc(ctypes.byref(g), 1.4, 1e-3, af.AF_TAI, ctypes.byref(st), ctypes.byref(st),
                      None)
    assert rc == af.AF_ERR_ARG


def test_noalloc_clears_a_flag_left_by_the_previous_call():
    """The work area keeps the last call's contents, its error word included.  A
    call whose time step is far above the acoustic CFL limit raises the
    device-side CFL flag (reported, not faulted); the next, valid call on the
    same stream must start from a clear error word and match the handle step."""
    torch = pytest.importorskip("torch")
    step_noalloc = _lib()
    P = I.random_smooth(16, 16, seed=1)
    n = P.grid.nx * P.grid.ny
    g = af.AfGrid(P.grid.nx, P.grid.ny, P.grid.h)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64")
    s.step(P.dt, 1)
    want = s.state()
    s.close()
    a = torch.from_numpy(P.state).cuda()
    b = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    rc = step_noalloc(ctypes.byref(g), P.gamma, 3.0 * P.dt, af.AF_TAI, ctypes.byref(_state(a, n)),
                      ctypes.byref(_state(b, n)), ctypes.c_void_p(stream))
    assert rc == af.AF_ERR_CFL
    rc = step_noalloc(ctypes.byref(g), P.gamma, P.dt, af.AF_TAI, ctypes.byref(_state(a, n)),
                      ctypes.byref(_state(b, n)), ctypes.c_void_p(stream))
    assert rc == af.AF_OK
    assert rel_linf(b.cpu().numpy(), want) < TOL64


def test_noalloc_rejects_overlapping_input_and_output():
    """`out` is written while later kernels of the step still read `in`."""
    torch = pytest.importorskip("torch")
    step_noalloc = _lib()
    nx = ny = 16
    g = af.AfGrid(nx, ny, 0.1)
    a = torch.ones((16, ny, nx), dtype=torch.float64, device="cuda")
    same = af._state_struct(a.data_ptr(), nx * ny)
    shifted = af._state_struct(a.data_ptr() + 8 * nx * ny, nx * ny)  # planes shifted by one
    for out in (same, shifted):
        rc = step_noalloc(ctypes.byref(g), 1.4, 1e-3, af.AF_TAI, ctypes.byref(same),
                          ctypes.byref(out), None)
        assert rc == af.AF_ERR_ARG
