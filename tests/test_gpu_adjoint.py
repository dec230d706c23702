"""The hand-written discrete adjoint of the step (af_adjoint_step) and the
checkpointed differentiable rollout built on it.

* one step: <A^T lam, v> against <lam, (S(x+eps v) - S(x-eps v)) / 2 eps> with the
  GPU forward step (FP64, both variants);
* an FP64 CPU adjoint: the transpose of the oracle's step Jacobian, assembled
  column by column by central differences of the oracle on a 6x6 grid,
  compared element by element with the GPU adjoint;
* a 20-step rollout with checkpoints every 7 steps: the gradient of the final
  kinetic energy against central differences along seeded directions (KH
  initial data), in FP64 and FP32.  The KH data put convective feet exactly on
  cell boundaries (v vanishes on grid columns), where the discrete map is only
  piecewise smooth; a seeded 1e-4 smooth perturbation moves them off so that
  central differences measure the derivative the adjoint computes.
"""
import numpy as np
import pytest

import paper_2605_12915_gb300 as af
from workloads import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    af._build.build()
    af.load()


def _step(s, x, dt):
    s.set_state(x)
    s.step(dt, 1)
    return s.state()


@pytest.mark.parametrize("variant", ["tai", "rb"])
def test_one_step_adjoint_dot_product(variant):
    P = I.random_smooth(24, 20, seed=13, amp=0.05)
    dt = P.dt * (0.6 if variant == "rb" else 1.0)
    rng = np.random.default_rng(5)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64", variant=variant)
    lam = rng.normal(size=P.state.shape)
    adj = s.adjoint(dt, lam)
    for trial in range(3):
        v = rng.normal(size=P.state.shape) * 0.1
        eps = 1e-6
        yp = _step(s, P.state + eps * v, dt)
        ym = _step(s, P.state - eps * v, dt)
        rhs = np.sum(lam * (yp - ym)) / (2 * eps)
        lhs = np.sum(adj * v)
        assert abs(lhs - rhs) <= 1e-7 * max(abs(rhs), 1.0), (trial, lhs, rhs)
    s.close()


def test_adjoint_matches_fp64_cpu_adjoint_of_the_oracle(orc):
    """Transpose of the oracle's one-step Jacobian (central differences, 6x6
    grid), applied to a dense random lambda and to sparse ones (unit vectors at
    seeded entries, and one 2x2 block of cells): with a sparse lambda most nodes
    of a row have no adjoint to scatter, the case where the scatter's merging of
    neighbouring nodes' record updates must fall back to single updates."""
    P = I.random_smooth(6, 6, seed=21, amp=0.05, h=1.0 / 6)
    x = P.state
    n = x.size
    eps = 1e-6
    rng = np.random.default_rng(8)
    jac = np.empty((n, n))  # jac[d] = d y / d x_d
    flat = x.reshape(-1)
    for d in range(n):
        xp = flat.copy()
        xm = flat.copy()
        xp[d] += eps
        xm[d] -= eps
        yp, _ = orc.step(xp.reshape(x.shape), P.grid.h, P.gamma, P.dt)
        ym, _ = orc.step(xm.reshape(x.shape), P.grid.h, P.gamma, P.dt)
        jac[d] = ((yp - ym) / (2 * eps)).reshape(-1)
    lams = [rng.normal(size=x.shape)]
    for d in rng.choice(n, size=6, replace=False):
        e = np.zeros(n)
        e[d] = 1.0
        lams.append(e.reshape(x.shape))
    block = np.zeros(x.shape)
    block[:, 2:4, 1:3] = rng.normal(size=(16, 2, 2))
    lams.append(block)
    s = af.Solver(P.grid, P.gamma, x, precision="fp64")
    for k, lam in enumerate(lams):
        cpu = jac @ lam.reshape(-1)
        gpu = s.adjoint(P.dt, lam).reshape(-1)
        err = np.max(np.abs(gpu - cpu)) / np.max(np.abs(cpu))
        assert err < 1e-7, (k, err)
    s.close()


def _rollout_grad(P, n_steps, every, precision):
    import torch
    from paper_2605_12915_gb300.autograd import kinetic_energy, rollout
    x0 = torch.from_numpy(P.state.copy()).cuda().requires_grad_(True)
    xn = rollout(x0, P.grid, P.gamma, P.dt, n_steps, every, precision)
    J = kinetic_energy(xn, P.grid.h)
    J.backward()
    return float(J.detach()), x0.grad.cpu().numpy()


def _ke_after(P, x, n_steps, precision):
    s = af.Solver(P.grid, P.gamma, x, precision=precision)
    s.step(P.dt, n_steps)
    y = s.state()
    s.close()
    return 0.5 * P.grid.h ** 2 * np.sum((y[1] ** 2 + y[2] ** 2) / y[0])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 2e-3)])
def test_rollout_gradient_matches_finite_differences(precision, tol):
    pytest.importorskip("torch")
    P = I.kelvin_helmholtz(n=32)
    Q = I.random_smooth(32, 32, seed=17, amp=0.05, flow=(0.0, 0.0), h=P.grid.h)
    P.state = P.state + 2e-3 * (Q.state - np.mean(Q.state, axis=(1, 2), keepdims=True))
    n_steps, every = 20, 7
    J, g = _rollout_grad(P, n_steps, every, precision)
    rng = np.random.default_rng(3)
    for trial in range(4):
        d = rng.normal(size=P.state.shape)
        d /= np.max(np.abs(d))
        eps = 1e-6 if precision == "fp64" else 1e-3
        # FD always in FP64: the reference derivative
        fd = (_ke_after(P, P.state + eps * d, n_steps, "fp64") -
              _ke_after(P, P.state - eps * d, n_steps, "fp64")) / (2 * eps)
        ad = float(np.sum(g * d))
        assert abs(ad - fd) <= tol * max(abs(fd), 1e-12), (precision, trial, ad, fd)


def _adjoint_with_env(P, lam, precision, env, variant="tai", dt=None):
    import os
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        s = af.Solver(P.grid, P.gamma, P.state, precision=precision, variant=variant)
        out = s.adjoint(P.dt if dt is None else dt, lam)
        s.close()
        return out
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
@pytest.mark.parametrize("variant", ["tai", "rb"])
@pytest.mark.parametrize("shape,ctas", [((64, 48), None), ((200, 168), "3")])
def test_fp32_adjoint_paths_match_fp64_adjoint(precision, variant, shape, ctas):
    """The FP32 adjoint on grids the persistent fused kernel accepts: the fused
    reverse sweep (each tile's step recomputed and its fluxes and point updates
    reversed in shared memory), the kernel-per-stage sweep on the fused
    kernel's stored intermediates (AF_ADJ_FUSED=0) and the unfused path
    (AF_PIPE=0) all agree with the FP64 adjoint to FP32 accuracy.  200 x 168
    on three CTAs steps each CTA through fourteen tiles, some staged by tensor
    copies."""
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=23 + nx, amp=0.05)
    dt = P.dt * (0.6 if variant == "rb" else 1.0)
    lam = np.random.default_rng(4).normal(size=P.state.shape)
    env = {"AF_PIPE": ctas} if ctas else {}
    ref = _adjoint_with_env(P, lam, "fp64", {}, variant, dt)
    scale = np.max(np.abs(ref))
    for name, e in (("fused", env), ("staged", dict(env, AF_ADJ_FUSED="0")),
                    ("unfused", {"AF_PIPE": "0"})):
        got = _adjoint_with_env(P, lam, precision, e, variant, dt)
        assert np.max(np.abs(got - ref)) / scale < 2e-5, name
