"""GPU parity: the CUDA step through the C ABI against the FP64 CPU oracle on the
same seeded inputs (element by element), plus FP32 against FP64, conservation,
determinism and error reporting.

Tolerances (relative L-inf, per plane: max |a - b| / max |b|):
  FP64 GPU vs oracle after up to 100 steps ...... 1e-12
  FP32 / FP32+compensated vs FP64 after 100 steps  2e-5
"""
import numpy as np
import pytest

import paper_2605_12915_gb300 as af
from workloads import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def rel_linf(a, b):
    num = np.max(np.abs(a - b), axis=(1, 2))
    den = np.maximum(np.max(np.abs(b), axis=(1, 2)), 1e-300)
    return float(np.max(num / den))


@pytest.fixture(scope="module", autouse=True)
def built():
    af._build.build()
    af.load()


def run_gpu(P, n_steps, precision="fp64", variant="tai", dt=None):
    s = af.Solver(P.grid, P.gamma, P.state, precision=precision, variant=variant)
    s.step(P.dt if dt is None else dt, n_steps)
    out = s.state()
    s.close()
    return out


def run_orc(orc, P, n_steps, variant=0, dt=None):
    st, fl = orc.run(P.state, P.grid.h, P.gamma, P.dt if dt is None else dt, n_steps, variant)
    assert fl == 0
    return st


@pytest.mark.parametrize("variant", ["tai", "rb"])
@pytest.mark.parametrize("shape", [(8, 8), (37, 29), (70, 33)])
def test_fp64_matches_oracle_random(orc, shape, variant):
    """Ragged sizes spanning several thread blocks; 20 steps."""
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=nx + ny, amp=0.06)
    dt = P.dt * (0.6 if variant == "rb" else 1.0)
    got = run_gpu(P, 20, "fp64", variant, dt)
    want = run_orc(orc, P, 20, 0 if variant == "tai" else 1, dt)
    assert rel_linf(got, want) < TOL64


@pytest.mark.parametrize("shape", [(3, 3), (4, 4), (5, 7)])
def test_tiny_grids_match_oracle(orc, shape):
    """Grids smaller than one tile and barely wider than the stencils' reach:
    the periodic wrap is taken several times inside one tile.  FP64 with the
    transported, additive and foot-centred point updates, and the fused FP32
    kernels, 3 steps each, against the oracle on the same state."""
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=7 * nx + ny, amp=0.03)
    runs = (("tai", 0, P.dt), ("rb", 1, 0.6 * P.dt), ("fc", 2, P.dt))
    for variant, ov, dt in runs:
        want = run_orc(orc, P, 3, ov, dt)
        err = rel_linf(run_gpu(P, 3, "fp64", variant, dt), want)
        assert err < TOL64, (shape, variant, err)
        if variant == "tai":
            for precision in ("fp32", "fp32_comp"):
                err32 = rel_linf(run_gpu(P, 3, precision), want)
                assert err32 < TOL32, (shape, precision, err32)


def test_fp64_matches_oracle_vortex_100_steps(orc):
    """Isentropic vortex, 32^2, CFL 0.4, 100 steps, FP64, transported update."""
    P = I.vortex(n=32)
    got = run_gpu(P, 100, "fp64")
    want = run_orc(orc, P, 100)
    err = rel_linf(got, want)
    print("vortex fp64 vs oracle rel Linf", err)
    assert err < TOL64


def test_vortex_against_the_exact_translate():
    """Isentropic vortex (Sec. 6.2) on the GPU against its exact solution, the
    initial vortex translated by the free stream, after 100 steps of the 32^2
    workload (t = 3.75) and at the same time on 64^2 (200 steps).  The
    oracle's errors on the same runs are 8.8e-3 (32^2) and 1.3e-3 (64^2) in the
    density average against a vortex depth of 0.48 (log2 ratio 2.8), and at
    most 2.3% of a plane's range on any plane at 32^2.  The tails of the vortex are not periodic on [-5,5]^2,
    which puts a floor near 1e-5 far below these errors."""
    P = I.vortex(n=32)
    T = 100 * P.dt
    errs = {}
    for n in (32, 64):
        Q = I.vortex(n=n)
        ns = int(round(T / Q.dt))
        got = run_gpu(Q, ns, "fp64", dt=T / ns)
        ex = I.vortex_exact(Q.grid, T)
        # per plane: max |error| over the plane's range of values
        errs[n] = np.max(np.abs(got - ex), axis=(1, 2)) / np.ptp(ex, axis=(1, 2))
        print("vortex %d^2 vs exact after t = %.3f: per plane max |error| / range %s"
              % (n, T, np.array2string(errs[n], precision=2)))
    assert np.max(errs[32]) < 3e-2, errs[32]  # oracle: 2.3e-2 at most
    order = np.log2(errs[32][0] / errs[64][0])
    print("density-average order 32 -> 64: %.2f" % order)
    assert order > 2.3, order


@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
def test_fp32_vs_fp64_vortex_100_steps(precision):
    P = I.vortex(n=32)
    a = run_gpu(P, 100, precision)
    b = run_gpu(P, 100, "fp64")
    err = rel_linf(a, b)
    print("vortex", precision, "vs fp64 rel Linf", err)
    assert err < TOL32


def test_pulse_512_one_step_matches_oracle(orc):
    """Gaussian pulse at its full size (512^2): one step, whole grid, FP64."""
    P = I.pulse(n=512)
    got = run_gpu(P, 1, "fp64")
    want = run_orc(orc, P, 1)
    assert rel_linf(got, want) < TOL64


@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
def test_pulse_512_fp32_vs_fp64_100_steps(precision):
    P = I.pulse(n=512)
    a = run_gpu(P, 100, precision)
    b = run_gpu(P, 100, "fp64")
    err = rel_linf(a, b)
    print("pulse", precision, "vs fp64 rel Linf", err)
    assert err < TOL32


def _mirror_x(st):
    """Reflection x -> -x on the symmetric grid [-L, L] with an even cell count."""
    out = np.empty_like(st)
    cell = lambda a: a[:, ::-1]
    vert = lambda a: np.roll(a[:, ::-1], 1, axis=1)
    for k in range(4):
        sgn = -1.0 if k == 1 else 1.0
        out[k] = sgn * cell(st[k])
        out[4 + k] = sgn * vert(st[4 + k])
        out[8 + k] = sgn * vert(st[8 + k])
        out[12 + k] = sgn * cell(st[12 + k])
    return out


def _swap_xy(st):
    """Reflection x <-> y: E_v and E_h exchange, u and v exchange."""
    out = np.empty_like(st)
    perm = [0, 2, 1, 3]
    for k in range(4):
        out[perm[k]] = st[k].T
        out[4 + perm[k]] = st[4 + k].T
        out[8 + perm[k]] = st[12 + k].T
        out[12 + perm[k]] = st[8 + k].T
    return out


def _pressure_at(st, wc, X, Y):
    """Q2 reconstruction of p at points (X, Y) in cell units (vectorised; the
    centre values wc come from the oracle's centre recovery)."""
    ny, nx = st.shape[1:]
    ci, cj = np.floor(X).astype(int), np.floor(Y).astype(int)
    L = lambda s: (0.5 * s * (s - 1), 1 - s * s, 0.5 * s * (s + 1))
    lx, ly = L(2 * (X - ci) - 1), L(2 * (Y - cj) - 1)
    i0, i1, j0, j1 = ci % nx, (ci + 1) % nx, cj % ny, (cj + 1) % ny
    V, Ev, Eh, C = st[7], st[11], st[15], wc[3]
    rows = [(V[j0, i0], Eh[j0, i0], V[j0, i1]), (Ev[j0, i0], C[j0, i0], Ev[j0, i1]),
            (V[j1, i0], Eh[j1, i0], V[j1, i1])]
    return sum(ly[b] * sum(lx[a] * rows[b][a] for a in range(3)) for b in range(3))


def _radial_error(orc, P, st):
    """max over radii r in [0.1, 0.9] of (max - min) of p over 256 angles."""
    wc, fl = orc.center_recovery(st, P.gamma)
    assert fl == 0
    th = np.linspace(0.0, 2 * np.pi, 256, endpoint=False)
    worst = 0.0
    for r in np.linspace(0.1, 0.9, 33):
        X = (r * np.cos(th) - P.grid.x0) / P.grid.h
        Y = (r * np.sin(th) - P.grid.y0) / P.grid.h
        p = _pressure_at(st, wc, X, Y)
        worst = max(worst, float(p.max() - p.min()))
    return worst


def test_pulse_512_400_steps_symmetry_and_fp32(orc):
    """The Gaussian pulse workload in full (512^2, 400 steps): the FP64 state keeps
    the grid's mirror and diagonal symmetry to rounding (measured 1e-14), its
    radial-symmetry error stays small (measured 6.9e-6 of the pulse's pressure
    amplitude), and both FP32 modes stay within 2e-5 of FP64 (measured 3.5e-6)."""
    P = I.pulse(n=512)
    amp = float(np.max(P.state[7]) - np.min(P.state[7]))
    b = run_gpu(P, 400, "fp64")
    scale = np.max(np.abs(b))
    assert np.max(np.abs(_mirror_x(b) - b)) / scale < 1e-13
    assert np.max(np.abs(_swap_xy(b) - b)) / scale < 1e-13
    rad = _radial_error(orc, P, b) / amp
    print("pulse 512^2, 400 steps: radial-symmetry error / amplitude", rad)
    assert rad < 1e-4
    for precision in ("fp32", "fp32_comp"):
        a = run_gpu(P, 400, precision)
        err = rel_linf(a, b)
        print("pulse 512^2, 400 steps,", precision, "vs fp64 rel Linf", err)
        assert err < TOL32


def test_free_stream(orc):
    P = I.uniform(33, 17)
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-6), ("fp32_comp", 1e-6)):
        out = run_gpu(P, 10, prec)
        assert rel_linf(out, P.state) < tol, prec


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32_comp", 1e-12)])
def test_conservation(precision, tol):
    P = I.random_smooth(64, 48, seed=5, amp=0.05)
    s = af.Solver(P.grid, P.gamma, P.state, precision=precision)
    inv0 = s.invariants()
    s.step(P.dt, 100)
    inv1 = s.invariants()
    s.close()
    scale = np.array([inv0[0], inv0[0], inv0[0], inv0[3]])
    drift = np.abs(inv1[:4] - inv0[:4]) / scale
    print(precision, "conservation drift", drift)
    assert np.all(drift < tol), drift


def test_invariants_match_oracle(orc):
    P = I.random_smooth(40, 24, seed=8, amp=0.05)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64")
    s.step(P.dt, 5)
    st = s.state()
    got = s.invariants()
    s.close()
    want = orc.invariants(st, P.grid.h, P.gamma)
    for k in range(10):
        assert abs(got[k] - want[k]) <= 1e-12 * max(abs(want[k]), 1.0), \
            (af.INVARIANT_NAMES[k], got[k], want[k])
    # the vorticity integral vanishes up to rounding on both sides
    assert abs(got[10]) < 1e-15 and abs(want[10]) < 1e-15


def test_deterministic():
    P = I.random_smooth(96, 64, seed=2)
    a = run_gpu(P, 10, "fp32_comp")
    b = run_gpu(P, 10, "fp32_comp")
    assert np.array_equal(a, b)


def test_errors_are_reported():
    P = I.random_smooth(16, 16, seed=1)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32")
    assert af.af_step(s.handle, P.dt * 3.0, 1) == af.AF_OK  # asynchronous
    assert af.af_sync(s.handle) == af.AF_ERR_CFL
    assert af.af_step(s.handle, P.dt, 1) == af.AF_ERR_CFL  # latched
    s.set_state(P.state)  # clears the latch
    assert af.af_step(s.handle, P.dt, 1) == af.AF_OK
    assert af.af_sync(s.handle) == af.AF_OK
    bad = P.state.copy()
    bad[7, 3, 4] = -1.0  # negative vertex pressure
    s.set_state(bad)
    af.af_step(s.handle, P.dt, 1)
    assert af.af_sync(s.handle) == af.AF_ERR_NONPHYSICAL
    s.close()
    assert af.af_step(0, 0.1, 1) == af.AF_ERR_ARG


def test_timed_out_wait_is_reported_and_the_handle_recovers(monkeypatch):
    """The bounded wait for a tile's tensor copies.  AF_TEST_LATE_WAIT=1 makes the
    first such wait of every CTA of the handle's first step give up at once (the
    copies are real and complete; the CTA drains them, flags the timeout and
    stops).  100 x 70 cells: 12 tiles, two of them staged by tensor copies.  The
    step must report AF_ERR_TIMEOUT, keep reporting it until the state is reset,
    and the next step after af_set_state must be bitwise the plain step."""
    P = I.random_smooth(100, 70, seed=5, amp=0.05)
    clean = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp")
    clean.step(P.dt, 1)
    want = clean.state()
    clean.close()
    monkeypatch.setenv("AF_TEST_LATE_WAIT", "1")
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp")
    monkeypatch.delenv("AF_TEST_LATE_WAIT")
    assert af.af_step(s.handle, P.dt, 1) == af.AF_OK  # asynchronous
    assert af.af_sync(s.handle) == af.AF_ERR_TIMEOUT
    assert af.af_step(s.handle, P.dt, 1) == af.AF_ERR_TIMEOUT  # latched
    s.set_state(P.state)  # clears the latch
    s.step(P.dt, 1)
    s.sync()
    assert np.array_equal(s.state(), want)
    s.close()


def test_device_tensors_and_stream():
    torch = pytest.importorskip("torch")
    P = I.random_smooth(48, 40, seed=3)
    st = torch.from_numpy(P.state).cuda()
    stream = torch.cuda.Stream()
    s = af.Solver(P.grid, P.gamma, st, precision="fp64", stream=stream)
    s.step(P.dt, 3)
    out = torch.empty_like(st)
    s.state(out)
    host = run_gpu(P, 3, "fp64")
    assert np.array_equal(out.cpu().numpy(), host)
    s.close()


def _with_env(name, value, fn):
    import os
    old = os.environ.get(name)
    os.environ[name] = value
    try:
        return fn()
    finally:
        if old is None:
            del os.environ[name]
        else:
            os.environ[name] = old


def _with_path(path, fn):
    return _with_env("AF_PATH", path, fn)


@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
@pytest.mark.parametrize("shape", [(8, 8), (70, 33), (97, 130)])
def test_fused_matches_unfused_path(precision, shape):
    """The fused single-pass kernel and the multi-kernel path compute the same step."""
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=11 + nx, amp=0.06)
    a = _with_path("fused", lambda: run_gpu(P, 20, precision))
    b = _with_path("ref", lambda: run_gpu(P, 20, precision))
    assert rel_linf(a, b) < 5e-6


@pytest.mark.parametrize("tma", ["1", "0"])
@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
@pytest.mark.parametrize("shape,ctas", [((40, 38), "1"), ((72, 44), "2"), ((100, 70), "3"),
                                        ((128, 160), "7"), ((424, 392), "")])
def test_pipelined_kernel_is_bitwise_the_per_tile_kernel(precision, shape, ctas, tma):
    """The persistent kernel (tiles stepped through by few CTAs, the next tile's
    input copied while the current one finishes) computes exactly what one CTA per
    tile computes, whether interior tiles are staged by tensor copies or, like the
    tiles on the periodic boundary, by cp.async (AF_TMA=0); (40, 38) is the
    smallest grid it accepts, and 424 x 392 (182 tiles, ragged in both directions)
    runs on the default one-wave grid."""
    nx, ny = shape
    P = I.random_smooth(nx, ny, seed=5 + nx, amp=0.06)

    def pipelined():
        if ctas:
            return _with_env("AF_PIPE", ctas, lambda: run_gpu(P, 10, precision))
        import os
        assert "AF_PIPE" not in os.environ
        return run_gpu(P, 10, precision)
    a = _with_env("AF_TMA", tma, pipelined)
    b = _with_env("AF_PIPE", "0", lambda: run_gpu(P, 10, precision))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("variant", ["tai", "rb"])
def test_fused_fp32_matches_oracle_random(orc, variant):
    P = I.random_smooth(70, 45, seed=4, amp=0.06)
    dt = P.dt * (0.6 if variant == "rb" else 1.0)
    got = _with_path("fused", lambda: run_gpu(P, 20, "fp32_comp", variant, dt))
    want = run_orc(orc, P, 20, 0 if variant == "tai" else 1, dt)
    assert rel_linf(got, want) < TOL32


@pytest.mark.parametrize("variant", ["tai", "rb"])
def test_pipelined_fp32_matches_oracle_random(orc, variant):
    """Persistent kernel with two CTAs over a 3 x 2 tile grid against the oracle."""
    P = I.random_smooth(76, 48, seed=9, amp=0.06)
    dt = P.dt * (0.6 if variant == "rb" else 1.0)
    got = _with_env("AF_PIPE", "2", lambda: run_gpu(P, 20, "fp32_comp", variant, dt))
    want = run_orc(orc, P, 20, 0 if variant == "tai" else 1, dt)
    assert rel_linf(got, want) < TOL32


def test_state_transfer_pinned_pageable_and_device_agree():
    """Pinned host planes are read and written in place by the conversion
    kernels, pageable ones through the staging copy; both give the same bits
    as device buffers (and AF_ZERO_COPY=0 forces the copies)."""
    import torch
    P = I.random_smooth(72, 40, seed=31, amp=0.06)
    for precision in ("fp64", "fp32_comp"):
        outs = []
        for kind in ("numpy", "pinned", "device", "copies"):
            def run():
                if kind == "numpy":
                    src = P.state.copy()
                elif kind == "pinned":
                    src = torch.from_numpy(P.state.copy()).pin_memory()
                else:
                    src = torch.from_numpy(P.state.copy()).cuda()
                s = af.Solver(P.grid, P.gamma, src, precision=precision)
                s.step(P.dt, 3)
                s.set_state(src)
                s.step(P.dt, 3)
                if kind == "pinned":
                    out = torch.empty(P.state.shape, dtype=torch.float64).pin_memory()
                    s.state(out)
                    out = out.numpy()
                elif kind == "device":
                    out = torch.empty(P.state.shape, dtype=torch.float64, device="cuda")
                    s.state(out)
                    out = out.cpu().numpy()
                else:
                    out = s.state()
                s.close()
                return out
            outs.append(_with_env("AF_ZERO_COPY", "0", run) if kind == "copies" else run())
        for o in outs[1:]:
            assert np.array_equal(outs[0], o), precision


def test_fused_conservation_and_determinism():
    P = I.random_smooth(130, 70, seed=6, amp=0.05)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp")
    inv0 = s.invariants()
    s.step(P.dt, 100)
    inv1 = s.invariants()
    a = s.state()
    s.close()
    drift = np.abs(inv1[:4] - inv0[:4]) / np.array([inv0[0], inv0[0], inv0[0], inv0[3]])
    assert np.all(drift < 1e-12), drift
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp")
    s.step(P.dt, 100)
    b = s.state()
    s.close()
    assert np.array_equal(a, b)


def test_reach_limit_is_flagged_not_faulted():
    """A velocity that carries the foot more than one cell is reported as a CFL error."""
    P = I.uniform(40, 40, u=9.0, v=0.1, p=0.2, h=0.1)
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32")
    dt = 1.5 * P.grid.h / 9.0  # |u| dt / h = 1.5; acoustic CFL stays below 1/2
    af.af_step(s.handle, dt, 1)
    assert af.af_sync(s.handle) == af.AF_ERR_CFL
    s.close()


def _window(state, ci, cj, w):
    """Periodic window of w x w cells whose lower-left cell is (ci, cj)."""
    ny, nx = state.shape[1:]
    ii = (ci + np.arange(w)) % nx
    jj = (cj + np.arange(w)) % ny
    return np.ascontiguousarray(state[:, jj][:, :, ii])


def test_full_size_shear_2048_windows_match_oracle(orc):
    """The benchmark workload at full size (2048^2 shear layer, FP32 with
    compensated averages, fused kernel): 10 GPU steps on the whole grid, against
    the FP64 oracle run on periodic 116^2 windows around sampled cells; the
    central 16^2 cells of each window lie beyond the 10-step dependence radius
    of the window's artificial boundary, so there the oracle is exact."""
    P = I.shear(n=2048)
    steps, margin, core = 10, 50, 16
    got = run_gpu(P, steps, "fp32_comp")
    scale = np.max(np.abs(P.state), axis=(1, 2))
    scale[[1, 2, 5, 6, 9, 10, 13, 14]] = np.maximum(scale[[1, 2, 5, 6, 9, 10, 13, 14]], 0.05)
    rng = np.random.default_rng(0)
    w = core + 2 * margin
    worst = 0.0
    for ci, cj in rng.integers(0, 2048, size=(6, 2)):
        win = _window(P.state, ci - margin, cj - margin, w)
        want, fl = orc.run(win, P.grid.h, P.gamma, P.dt, steps)
        assert fl == 0
        want_core = want[:, margin:margin + core, margin:margin + core]
        got_core = _window(got, ci, cj, core)
        err = np.max(np.abs(got_core - want_core), axis=(1, 2)) / scale
        worst = max(worst, float(np.max(err)))
    print("2048^2 window parity, FP32 vs FP64 oracle, rel Linf", worst)
    assert worst < TOL32


@pytest.mark.parametrize("precision", ["fp64", "fp32_comp"])
def test_exchange_is_get_then_set(precision):
    """af_exchange_state = af_get_state then af_set_state, bitwise, for pinned
    and pageable host planes and device planes; overlapping planes are refused."""
    import torch
    P = I.random_smooth(70, 44, seed=41, amp=0.05)
    Q = I.random_smooth(70, 44, seed=42, amp=0.05)
    ref = af.Solver(P.grid, P.gamma, P.state, precision=precision)
    ref.step(P.dt, 3)
    want_out = ref.state()
    ref.set_state(Q.state)
    ref.step(Q.dt, 2)
    want_next = ref.state()
    ref.close()
    pinned_in = torch.from_numpy(Q.state.copy()).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    cases = [("pinned", pinned_out, pinned_in),
             ("pageable", np.empty_like(Q.state), Q.state.copy()),
             ("device", torch.empty(Q.state.shape, dtype=torch.float64, device="cuda"),
              torch.from_numpy(Q.state.copy()).cuda())]
    for name, out, new in cases:
        s = af.Solver(P.grid, P.gamma, P.state, precision=precision)
        s.step(P.dt, 3)
        s.exchange(out, new)
        s.step(Q.dt, 2)
        s.sync()  # host `out` may still be arriving until a call other than step
        got = out.cpu().numpy() if hasattr(out, "cpu") else out
        assert np.array_equal(got, want_out), name
        assert np.array_equal(s.state(), want_next), name
        with pytest.raises(af.AfError):
            s.exchange(new, new)
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_comp"])
def test_exchange_async_streams_like_the_synchronous_exchange(precision):
    """af_exchange_state_async: a stream of distinct inputs, each stepped once
    and handed out by the next call (both staging buffers of each direction in
    turn), gives bitwise the one-step results of the inputs, for pinned and
    pageable host planes; a chain where one call's output is the next call's
    input, and an output buffer reused while its copy may be in flight, gives
    the synchronous exchange's results; overlapping planes are refused."""
    import torch
    X = [I.random_smooth(68, 40, seed=50 + k, amp=0.05) for k in range(5)]
    dt = 0.9 * min(P.dt for P in X)  # one time step for every input
    ref = af.Solver(X[0].grid, X[0].gamma, X[0].state, precision=precision)
    want = []
    for P in X:
        ref.set_state(P.state)
        ref.step(dt, 1)
        want.append(ref.state())
    ref.close()
    for kind in ("pinned", "pageable"):
        if kind == "pinned":
            ins = [torch.from_numpy(P.state.copy()).pin_memory() for P in X]
            outs = [torch.empty_like(ins[0]).pin_memory() for _ in X]
        else:
            ins = [P.state.copy() for P in X]
            outs = [np.empty_like(X[0].state) for _ in X]
        s = af.Solver(X[0].grid, X[0].gamma, X[0].state, precision=precision)
        s.set_state(ins[0])
        for k in range(4):
            s.step(dt, 1)
            s.exchange_async(outs[k], ins[k + 1])
        s.step(dt, 1)
        s.sync()
        for k in range(4):
            got = outs[k].numpy() if hasattr(outs[k], "numpy") else outs[k]
            assert np.array_equal(got, want[k]), (kind, k)
        assert np.array_equal(s.state(), want[4]), kind
        with pytest.raises(af.AfError):
            s.exchange_async(ins[0], ins[0])
        s.close()
    # chained buffers, as in the synchronous chain below: the same calls through
    # both exchanges give the same bits (a state taken back in has made the
    # round trip through its FP64 planes on both paths)
    P, Q = X[0], X[1]

    def chain(exchange_name):
        A = torch.empty(P.state.shape, dtype=torch.float64).pin_memory()
        B = torch.from_numpy(Q.state.copy()).pin_memory()
        C = torch.empty_like(A).pin_memory()
        s = af.Solver(P.grid, P.gamma, P.state, precision=precision)
        exchange = getattr(s, exchange_name)
        s.step(dt, 1)
        exchange(A, B)  # A <- S1 (in flight), state <- Q
        exchange(C, A)  # C <- Q, state <- A = S1 once it has arrived
        s.step(dt, 1)
        exchange(C, B)  # C <- S2 while the previous copy into C may be in flight
        s.sync()
        out = (A.numpy().copy(), C.numpy().copy(), s.state())
        s.close()
        return out

    for got, want_ in zip(chain("exchange_async"), chain("exchange")):
        assert np.array_equal(got, want_)


@pytest.mark.parametrize("precision", ["fp64", "fp32_comp"])
def test_exchange_chain_through_pinned_buffers(precision):
    """Streaming through host buffers: the state handed out by one exchange is
    taken back in by the next (whose incoming copy must wait for that outgoing
    one), while the same output buffer is reused."""
    import torch
    P = I.random_smooth(64, 40, seed=43, amp=0.05)
    Q = I.random_smooth(64, 40, seed=44, amp=0.05)
    ref = af.Solver(P.grid, P.gamma, P.state, precision=precision)
    ref.set_state(Q.state)
    q_round = ref.state()  # Q through the working precision
    ref.set_state(P.state)
    ref.step(P.dt, 1)
    s1 = ref.state()
    ref.step(P.dt, 1)
    s2 = ref.state()
    ref.close()
    A = torch.empty(P.state.shape, dtype=torch.float64).pin_memory()
    B = torch.from_numpy(Q.state.copy()).pin_memory()
    C = torch.empty_like(A).pin_memory()
    s = af.Solver(P.grid, P.gamma, P.state, precision=precision)
    s.step(P.dt, 1)
    s.exchange(A, B)  # A <- S1 (in flight), state <- Q
    s.exchange(C, A)  # C <- Q, state <- A = S1 once it has arrived
    s.step(P.dt, 1)
    s.exchange(C, B)  # C <- S2, reused while the previous copy into it may be in flight
    s.sync()
    assert np.array_equal(A.numpy(), s1)
    assert np.array_equal(C.numpy(), s2)
    assert np.array_equal(s.state(), q_round)
    # a longer stream: each step's result out, the same input back in, the
    # outputs alternating between two buffers (both export buffers in turn)
    outs = [torch.empty_like(A).pin_memory() for _ in range(2)]
    src = torch.from_numpy(P.state.copy()).pin_memory()
    s.set_state(src)
    for i in range(5):
        s.step(P.dt, 1)
        s.exchange(outs[i % 2], src)
    s.sync()
    assert np.array_equal(outs[0].numpy(), s1) and np.array_equal(outs[1].numpy(), s1)
    s.close()
