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


N_DIRECTIONS = 64  # the workload's seeded directions


@pytest.fixture(scope="module")
def kh_differences(kh_full):
    """Central differences (FP64 GPU step, eps 1e-7) of J after LINEAR_STEPS
    steps along N_DIRECTIONS seeded smooth directions: (directions, values)."""
    P = kh_full
    eps = 1e-7
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64")

    def J(x):
        s.set_state(x)
        s.step(P.dt, LINEAR_STEPS)
        return _ke(s.state(), P.grid.h)

    dirs, fds = [], []
    for seed in range(2000, 2000 + N_DIRECTIONS):
        d = I.smooth_direction(P.grid, seed)
        dirs.append(seed)
        fds.append((J(P.state + eps * d) - J(P.state - eps * d)) / (2 * eps))
    s.close()
    return dirs, fds


# Each direction's error |adjoint - difference| is stated relative to the
# largest |difference| over the directions: some seeded directions are nearly
# orthogonal to the gradient, and their own difference is then too small to
# normalise by.  The FP32 adjoint is linearised about the FP32 trajectory, which
# near the sheet already departs from the FP64 one at 100 steps (the FP32 and
# FP64 gradients differ there by up to 2e-3 of max |g|), hence 1e-4 for FP32;
# FP64 1e-6.
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-6)])
def test_kh_1024_gradient_matches_differences_in_linear_regime(kh_full, kh_differences,
                                                               precision, tol):
    P = kh_full
    _, _, g = _rollout(P, LINEAR_STEPS, EVERY, precision)
    seeds, fds = kh_differences
    fds = np.array(fds)
    ads = np.array([float(np.sum(g * I.smooth_direction(P.grid, seed))) for seed in seeds])
    err = np.abs(ads - fds) / np.max(np.abs(fds))
    own = np.abs(ads - fds) / np.abs(fds)
    print(f"KH 1024^2, {LINEAR_STEPS} steps, {precision}, {len(seeds)} directions: adjoint vs "
          f"central differences, max error / max |difference| {err.max():.2e}; relative to "
          f"each direction's own difference: median {np.median(own):.2e}, max {own.max():.2e} "
          f"(|difference| from {np.min(np.abs(fds)):.2e} to {np.max(np.abs(fds)):.2e})")
    assert err.max() <= tol, err


def test_kh_1024_full_rollout_gradient(kh_full):
    """The full 1000-step horizon in FP32 with compensated averages (the
    benchmark's precision).  With the time step fixed by CFL 0.4 on the initial
    state, the flow's wave speed grows: max(|u| + c) dt / h rises from 0.40 to
    0.51-0.52 by step 1000 in every precision (measured), so the acoustic limit
    c dt / h <= 1/2 of the exact acoustic operator is approached, and which
    trajectory crosses it depends on rounding (the perturbed plain-FP32 one does,
    near step 700, and is stopped by AF_ERR_CFL as designed)."""
    P = kh_full
    xn, J, g50 = _rollout(P, STEPS_FULL, EVERY, "fp32_comp")
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp")
    s.step(P.dt, STEPS_FULL)
    plain = s.state()
    s.close()
    assert np.array_equal(xn, plain), "the rollout's forward pass is the plain step"
    assert np.isfinite(J) and np.isfinite(g50).all()
    h2 = P.grid.h ** 2
    growth = np.abs(g50).max() / h2
    # the reason the difference check stops at LINEAR_STEPS
    assert growth > 1e3, growth
    _, J40, g40 = _rollout(P, STEPS_FULL, 40, "fp32_comp")
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


def _rel_per_plane(a, b):
    num = np.max(np.abs(a - b), axis=(1, 2))
    den = np.maximum(np.max(np.abs(b), axis=(1, 2)), 1e-300)
    return float(np.max(num / den))


def _fp64_run(P, x0):
    s = af.Solver(P.grid, P.gamma, x0, precision="fp64")
    s.step(P.dt, 50)
    y50 = s.state()
    s.step(P.dt, 50)
    y100 = s.state()
    s.close()
    return y50, y100


def test_kh_1024_fp32_vs_fp64_against_its_conditioning():
    """FP32 against FP64 on the workload's own (unperturbed) data, next to the
    workload's conditioning: FP64 from initial data perturbed at the FP32
    rounding level, (a) every value multiplied by 1 + 2^-24 r with r seeded
    uniform in [-1, 1], (b) every value rounded to float32 and back, against
    FP64 from the exact data.  The distances are stated in both norms (per
    plane, and per field with velocity and momentum as vectors).

    The difference sits on the rows of the two vortex sheets and grows there
    about 12x every 50 steps from step 50 on, for the FP32 modes and for the
    perturbed FP64 runs alike: the grid-scale Kelvin-Helmholtz growth of the
    unresolved sheets amplifies any perturbation at rounding level.  FP32
    rounds its stored state at every step, not once, so its difference is a
    small multiple of that of one perturbation of the initial data.  The test
    asserts that multiple (at most 4 after 100 steps, in either norm) instead
    of the fixed 2e-5 that the smooth workloads meet; away from the sheets
    (more than 48 rows) and after 50 steps the 2e-5 bound holds as it is."""
    from bench import rel_linf_fields
    P = I.kelvin_helmholtz(n=N_FULL)
    sheet = np.minimum(np.abs(np.arange(N_FULL) - N_FULL // 4),
                       np.abs(np.arange(N_FULL) - 3 * N_FULL // 4))
    far = sheet > 48
    b50, b100 = _fp64_run(P, P.state)
    rng = np.random.default_rng(4242)
    pert = {"relative 2^-24": P.state * (1.0 + 2.0 ** -24 * rng.uniform(-1, 1, P.state.shape)),
            "float32 round trip": P.state.astype(np.float32).astype(np.float64)}
    cond = {}
    for name, x0 in pert.items():
        c50, c100 = _fp64_run(P, x0)
        cond[name] = (rel_linf_fields(c100, b100), _rel_per_plane(c100, b100))
        print(f"KH 1024^2 fp64 ({name} perturbation) vs fp64: 50 steps "
              f"{rel_linf_fields(c50, b50):.2e} / {_rel_per_plane(c50, b50):.2e}, 100 steps "
              f"{cond[name][0]:.2e} / {cond[name][1]:.2e} (per field / per plane)")
    ref_field = max(c[0] for c in cond.values())
    ref_plane = max(c[1] for c in cond.values())
    for precision in ("fp32", "fp32_comp"):
        s = af.Solver(P.grid, P.gamma, P.state, precision=precision)
        s.step(P.dt, 50)
        a50 = s.state()
        s.step(P.dt, 50)
        a100 = s.state()
        s.close()
        e50, e100 = rel_linf_fields(a50, b50), rel_linf_fields(a100, b100)
        p50, p100 = _rel_per_plane(a50, b50), _rel_per_plane(a100, b100)
        efar = rel_linf_fields(a100[:, far], b100[:, far])
        print(f"KH 1024^2 {precision} vs fp64: 50 steps {e50:.2e} / {p50:.2e}, 100 steps "
              f"{e100:.2e} / {p100:.2e} (per field / per plane), 100 steps away from the "
              f"sheets {efar:.2e}; ratio to the rounding-level perturbation "
              f"{e100 / ref_field:.2f} / {p100 / ref_plane:.2f}")
        assert e50 < 2e-5 and efar < 2e-5
        assert e100 <= 4 * ref_field and p100 <= 4 * ref_plane
