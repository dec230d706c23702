"""The bounds-checking debug build: the same CUDA sources compiled with
AF_BOUNDS_CHECK, where the fused step checks its shared-memory indices (foot
cells, stencil and node cells, point, edge and flux indices) against their
regions and reports a violation as AF_ERR_BOUNDS instead of touching memory
outside them.  On every path the fused kernels take -- the one-CTA-per-tile
kernel on tiny and ragged grids, the persistent kernel staging by tensor copies
and by cp.async, feet clamped at the one-cell reach, the adjoint's fused
reverse sweep -- no check may fire, and the forward results must be bitwise
those of the regular library (the checks only read indices)."""
import contextlib
import ctypes
import os

import numpy as np
import pytest

import paper_2605_12915_gb300 as af
from paper_2605_12915_gb300 import _build
from workloads import inputs as I

pytestmark = pytest.mark.gpu

CHECK_LIB = os.path.join(os.path.dirname(_build.LIB), "libaf_check.so")
_FUNCS = ["af_init", "af_step", "af_sync", "af_get_state", "af_set_state", "af_adjoint_step",
          "af_reduce_invariants", "af_destroy", "af_status_string"]


@pytest.fixture(scope="module")
def checked():
    regular = af.load()
    _build.build(out=CHECK_LIB, extra_flags=["-DAF_BOUNDS_CHECK"])
    lib = ctypes.CDLL(CHECK_LIB)
    for name in _FUNCS:
        getattr(lib, name).argtypes = getattr(regular, name).argtypes
        getattr(lib, name).restype = getattr(regular, name).restype
    return lib


@contextlib.contextmanager
def using(lib):
    """The binding's calls go to `lib` inside the block."""
    saved = af._lib
    af._lib = lib
    try:
        yield
    finally:
        af._lib = saved


def _run(P, precision, variant, n_steps, dt=None):
    s = af.Solver(P.grid, P.gamma, P.state, precision=precision, variant=variant)
    s.step(P.dt if dt is None else dt, n_steps)
    s.sync()  # raises on any latched status, AF_ERR_BOUNDS included
    out = s.state()
    s.close()
    return out


@pytest.mark.parametrize("shape,precision,variant,tma", [
    ((5, 7), "fp32_comp", "tai", "1"),      # one CTA per tile, wrapped several times
    ((37, 29), "fp32", "rb", "1"),          # one CTA per tile, ragged edges
    ((100, 70), "fp32_comp", "tai", "1"),   # persistent: tensor copies inside, cp.async on the wrap
    ((100, 70), "fp32_comp", "rb", "1"),
    ((72, 44), "fp32", "tai", "0"),         # persistent, every tile by cp.async
])
def test_checked_build_is_silent_and_bitwise(checked, monkeypatch, shape, precision, variant, tma):
    monkeypatch.setenv("AF_TMA", tma)
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=nx + 3 * ny, amp=0.06)
    dt = P.dt * (0.6 if variant == "rb" else 1.0)
    want = _run(P, precision, variant, 3, dt)
    with using(checked):
        got = _run(P, precision, variant, 3, dt)
    assert np.array_equal(got, want)


def test_checked_build_clamped_feet_report_cfl_only(checked):
    """Feet carried beyond one cell are clamped to the reach before any index is
    formed: the step reports AF_ERR_CFL, never AF_ERR_BOUNDS."""
    P = I.uniform(40, 40, u=9.0, v=0.1, p=0.2, h=0.1)
    with using(checked):
        s = af.Solver(P.grid, P.gamma, P.state, precision="fp32")
        assert af.af_step(s.handle, 1.5 * P.grid.h / 9.0, 1) == af.AF_OK
        assert af.af_sync(s.handle) == af.AF_ERR_CFL
        s.close()


def test_checked_build_adjoint_sweep_is_silent(checked):
    """The adjoint's fused sweep recomputes each tile's step with the same
    checked code (its atomics make it order-dependent, so no bitwise check)."""
    P = I.random_smooth(100, 70, seed=9, amp=0.05)
    lam = np.random.default_rng(1).normal(size=P.state.shape)
    with using(checked):
        s = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp")
        out = s.adjoint(P.dt, lam)
        s.close()
    assert np.isfinite(out).all()
