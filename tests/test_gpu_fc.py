"""GPU parity of the foot-centred exact acoustic update (Appendix C, FP64):
the CUDA kernels (primitives by closed forms and projected-radius slicing,
inclusion-exclusion) against the FP64 CPU oracle (direct polar quadrature of
each fragment) on the same seeded inputs, element by element, relative L-inf
per plane 1e-12; plus the properties that hold at any size."""
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


@pytest.fixture(scope="module", autouse=True)
def built():
    af._build.build()
    af.load()


def run_gpu(P, n_steps, variant="fc", dt=None):
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64", variant=variant)
    s.step(P.dt if dt is None else dt, n_steps)
    out = s.state()
    s.close()
    return out


@pytest.mark.parametrize("shape,steps", [((8, 8), 4), ((37, 29), 2), ((70, 33), 1)])
def test_fc_matches_oracle_random(orc, shape, steps):
    """Seeded random smooth states with a mean flow: ragged sizes spanning
    several thread blocks, feet in every direction."""
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=nx * ny, amp=0.06)
    got = run_gpu(P, steps)
    want, fl = orc.run(P.state, P.grid.h, P.gamma, P.dt, steps, orc.FC)
    assert fl == 0
    err = rel_linf(got, want)
    print("foot-centred %dx%d, %d steps: GPU vs oracle %.2e" % (nx, ny, steps, err))
    assert err < TOL64


def test_fc_vortex_matches_oracle(orc):
    """Isentropic vortex 32^2 (CFL 0.4, total footprint below h/2), 5 steps."""
    P = I.vortex(n=32)
    got = run_gpu(P, 5)
    want, fl = orc.run(P.state, P.grid.h, P.gamma, P.dt, 5, orc.FC)
    assert fl == 0
    err = rel_linf(got, want)
    print("foot-centred vortex 32^2, 5 steps: GPU vs oracle %.2e" % err)
    assert err < TOL64


def test_fc_at_rest_is_the_transported_step():
    """A pulse at rest: in its first step every foot is its point, so the
    foot-centred step is the transported one (later steps move the fluid)."""
    P = I.pulse(n=40, amp=0.1, width2=0.05)
    a = run_gpu(P, 1, "fc")
    b = run_gpu(P, 1, "tai")
    assert rel_linf(a, b) < 1e-13


def test_fc_free_stream_conservation_and_footprint():
    U = I.uniform(24, 20)
    out = run_gpu(U, 2)
    assert np.max(np.abs(out - U.state)) < 1e-13
    P = I.random_smooth(48, 40, seed=2, amp=0.05)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64", variant="fc")
    inv0 = s.invariants()
    s.step(P.dt, 5)
    s.sync()
    inv1 = s.invariants()
    assert np.max(np.abs(inv1[:4] - inv0[:4]) / np.abs(inv0[:4])) < 1e-13
    # a time step that breaks the compact footprint is reported, not faulted
    assert af.af_step(s.handle, 1.4 * P.dt, 1) == af.AF_OK
    assert af.af_sync(s.handle) == af.AF_ERR_CFL
    s.close()


def test_fc_has_no_adjoint_and_no_fp32():
    P = I.random_smooth(16, 16, seed=4)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64", variant="fc")
    lam = np.ones_like(P.state)
    out = np.empty_like(lam)
    assert af.af_adjoint_step(s.handle, P.dt, lam, out) == af.AF_ERR_ARG
    s.close()
    with pytest.raises(af.AfError):
        af.Solver(P.grid, P.gamma, P.state, precision="fp32", variant="fc")
