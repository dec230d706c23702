"""The adjoint on the compressible Kelvin-Helmholtz workload at its full size:
[0,1]^2, 1024^2 cells, rho = 2 / 1, u = +-0.5, p = 2.5, v = 0.01 sin(4 pi x),
CFL 0.4, 1000 steps with a checkpoint every 50, J = the kinetic energy of the
final averages; and on a 32^2 copy of it against the FP64 CPU oracle.

The KH data put convective feet exactly on cell boundaries (v vanishes on grid
columns), where the discrete map is only piecewise smooth; a seeded smooth
2e-3 perturbation moves them off.  Directions are seeded smooth fields.

What the workload allows: up to about 100 steps the rollout is in its linear
regime and central differences converge (FP64 step, eps 1e-7); there the
gradient is checked against them.  Beyond that the vortex sheet's grid-scale
Kelvin-Helmholtz instability takes over: max |dJ/dx| / h^2 grows from 0.5 at
100 steps to about 6e2 at 200, 2e6 at 400 and 8e7 at 1000 steps, and a
perturbation of the initial data, whether eps d or FP64 rounding, is amplified
by the same factor, so that central differences over 1000 steps do not
converge for any eps.  The 1000-step gradient is therefore checked by
properties that need no differences: the rollout's forward state is bitwise the
plain step's, the gradient is finite, and it does not depend on the checkpoint
interval beyond the rounding of the adjoint's atomic sums.
"""
import numpy as np
import pytest

import paper_2605_12915_gb300 as af
from workloads import inputs as I

pytestmark = pytest.mark.gpu

N_FULL, STEPS_FULL, EVERY = 1024, 1000, 50
LINEAR_STEPS = 100  # two checkpoint segments, inside the linear regime


@pytest.fixture(scope="module", autouse=True)
def built():
    af._build.build()
    af.load()


def _perturbed_kh(n):
    P = I.kelvin_helmholtz(n=n)
    P.state = P.state + 2e-3 * I.smooth_direction(P.grid, 1000)
    return P


@pytest.fixture(scope="module")
def kh_full():
    return _perturbed_kh(N_FULL)


def _rollout(P, n_steps, every, precision):
    """(final state, J, dJ/dx0) through the checkpointed autograd rollout."""
    import torch
    from paper_2605_12915_gb300.autograd import kinetic_energy, rollout
    x0 = torch.from_numpy(P.state.copy()).cuda().requires_grad_(True)
    xn = rollout(x0, P.grid, P.gamma, P.dt, n_steps, every, precision)
    J = kinetic_energy(xn, P.grid.h)
    J.backward()
    return xn.detach().cpu().numpy(), float(J.detach()), x0.grad.cpu().numpy()


def _ke(state, h):
    return 0.5 * h * h * np.sum((state[1] ** 2 + state[2] ** 2) / state[0])


def _ke_gpu_fp64(P, x, n_steps):
    s = af.Solver(P.grid, P.gamma, x, precision="fp64")
    s.step(P.dt, n_steps)
    y = s.state()
    s.close()
    return _ke(y, P.grid.h)


# The FP32 adjoint is linearised about the FP32 trajectory, which near the sheet
# already departs from the FP64 one at 100 steps (the FP32 and FP64 gradients
# differ there by up to 2e-3 of max |g|); the measured directional error is
# 2e-5, hence 1e-4.  FP64: measured 1.1e-7.
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-6)])
def test_kh_1024_gradient_matches_differences_in_linear_regime(kh_full, precision, tol):
    P = kh_full
    _, _, g = _rollout(P, LINEAR_STEPS, EVERY, precision)
    eps = 1e-7
    worst = 0.0
    for seed in (2000, 2001, 2002):
        d = I.smooth_direction(P.grid, seed)
        fd = (_ke_gpu_fp64(P, P.state + eps * d, LINEAR_STEPS) -
              _ke_gpu_fp64(P, P.state - eps * d, LINEAR_STEPS)) / (2 * eps)
        ad = float(np.sum(g * d))
        rel = abs(ad - fd) / abs(fd)
        worst = max(worst, rel)
        assert rel <= tol, (precision, seed, ad, fd, rel)
    print(f"KH 1024^2, {LINEAR_STEPS} steps, {precision}: adjoint vs central differences {worst:.2e}")


def test_kh_1024_full_rollout_gradient(kh_full):
    P = kh_full
    xn, J, g50 = _rollout(P, STEPS_FULL, EVERY, "fp32")
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32")
    s.step(P.dt, STEPS_FULL)
    plain = s.state()
    s.close()
    assert np.array_equal(xn, plain), "the rollout's forward pass is the plain step"
    assert np.isfinite(J) and np.isfinite(g50).all()
    h2 = P.grid.h ** 2
    growth = np.abs(g50).max() / h2
    # the reason the difference check stops at LINEAR_STEPS
    assert growth > 1e3, growth
    _, J40, g40 = _rollout(P, STEPS_FULL, 40, "fp32")
    assert J40 == J
    rel = np.abs(g40 - g50).max() / np.abs(g50).max()
    dot = abs(np.sum(g40 * g50)) / np.sqrt(np.sum(g40 ** 2) * np.sum(g50 ** 2))
    print(f"KH 1024^2, {STEPS_FULL} steps: max|g|/h^2 {growth:.3e}, "
          f"checkpoints 50 vs 40: max diff {rel:.2e} of max|g|, cosine {dot:.9f}")
    assert rel <= 1e-2, rel


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-7)])
def test_kh_32_copy_gradient_matches_oracle_differences(orc, kh_full, precision, tol):
    """A 32^2 copy run to the same final time as the 1000-step full-size run."""
    P = _perturbed_kh(32)
    n_steps = int(round(STEPS_FULL * kh_full.dt / P.dt))
    _, _, g = _rollout(P, n_steps, EVERY, precision)
    eps = 1e-6
    worst = 0.0
    for seed in (3000, 3001, 3002, 3003):
        d = I.smooth_direction(P.grid, seed)
        yp, fp = orc.run(P.state + eps * d, P.grid.h, P.gamma, P.dt, n_steps)
        ym, fm = orc.run(P.state - eps * d, P.grid.h, P.gamma, P.dt, n_steps)
        assert fp == 0 and fm == 0
        fd = (_ke(yp, P.grid.h) - _ke(ym, P.grid.h)) / (2 * eps)
        ad = float(np.sum(g * d))
        rel = abs(ad - fd) / abs(fd)
        worst = max(worst, rel)
        assert rel <= tol, (precision, seed, ad, fd, rel)
    print(f"KH 32^2 copy, {n_steps} steps, {precision}: adjoint vs oracle differences {worst:.2e}")


def test_kh_1024_fp32_vs_fp64(kh_full):
    """FP32 against FP64 on the workload's own (unperturbed) data.  The difference
    sits on the rows of the two vortex sheets and grows there by about 12x every
    50 steps from step 50 on (the growth the gradient shows): 3.5e-6 after 50
    steps, 4.0e-5 (FP32) and 2.8e-5 (FP32 compensated) after 100 in the
    per-field form.  Away from the sheets (more than 48 rows) it stays at the
    level of the smooth workloads."""
    from bench import rel_linf_fields
    P = I.kelvin_helmholtz(n=N_FULL)
    sheet = np.minimum(np.abs(np.arange(N_FULL) - N_FULL // 4),
                       np.abs(np.arange(N_FULL) - 3 * N_FULL // 4))
    far = sheet > 48
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64")
    s.step(P.dt, 50)
    b50 = s.state()
    s.step(P.dt, 50)
    b100 = s.state()
    s.close()
    for precision in ("fp32", "fp32_comp"):
        s = af.Solver(P.grid, P.gamma, P.state, precision=precision)
        s.step(P.dt, 50)
        a50 = s.state()
        s.step(P.dt, 50)
        a100 = s.state()
        s.close()
        e50, e100 = rel_linf_fields(a50, b50), rel_linf_fields(a100, b100)
        efar = rel_linf_fields(a100[:, far], b100[:, far])
        print(f"KH 1024^2 {precision} vs fp64 (per field): 50 steps {e50:.2e}, "
              f"100 steps {e100:.2e}, 100 steps away from the sheets {efar:.2e}")
        assert e50 < 2e-5 and efar < 2e-5
        assert e100 < 1e-4
