"""Pins of the oracle's whole step (Sec. 6.1) against what the paper and the
mathematics fix: free-stream preservation (Sec. 4), conservation of the flux
difference update (Sec. 3.1), the exact frozen evolution when the generators
commute (Sec. 4.1), third- vs second-order one-step point accuracy of RB-TAI vs
RB on the linearized wave packet (Sec. 4.2, Sec. 5), isentropic-vortex
convergence (Sec. 6.2), grid symmetry of a radial pulse (Sec. 6.3), and the
Simpson inversion / Q2 interpolation building blocks (Sec. 2).
"""
import numpy as np
import pytest

from workloads import inputs as I

EPS = 1e-6


def test_free_stream_is_preserved(orc):
    P = I.uniform(9, 7, rho=1.3, u=0.4, v=-0.25, p=0.8)
    for variant in (orc.TAI, orc.RB):
        st, fl = orc.run(P.state, P.grid.h, P.gamma, P.dt, 5, variant)
        assert fl == 0
        assert np.max(np.abs(st - P.state) / np.abs(P.state).max(axis=(1, 2))[:, None, None]) < 1e-14


@pytest.mark.parametrize("variant", [0, 1])
def test_conservation_to_roundoff(orc, variant):
    P = I.random_smooth(20, 16, seed=3, amp=0.05)
    inv0 = orc.invariants(P.state, P.grid.h, P.gamma)
    st, fl = orc.run(P.state, P.grid.h, P.gamma, P.dt * (0.6 if variant else 1.0), 30, variant)
    assert fl == 0
    inv1 = orc.invariants(st, P.grid.h, P.gamma)
    scale = np.array([inv0[0], inv0[0], inv0[0], inv0[3]])
    drift = np.abs(inv1[:4] - inv0[:4]) / scale
    assert np.all(drift < 1e-13), drift
    # the point values changed: the test is not vacuous
    assert np.max(np.abs(st - P.state)) > 1e-4


def test_vorticity_integral_vanishes(orc):
    P = I.random_smooth(16, 16, seed=4, amp=0.08)
    st, _ = orc.run(P.state, P.grid.h, P.gamma, P.dt, 10)
    assert abs(orc.invariants(st, P.grid.h, P.gamma)[10]) < 1e-15


@pytest.mark.parametrize("variant", [0, 1])
def test_frozen_advection_is_exact(orc, variant):
    """Constant p and velocity: the acoustic increments vanish, RB == RB-TAI, and with
    u dt = h/2 the full-step foot of every point lands on a Q2 node, so the point
    values are shifted copies of the old ones (Sec. 4.1, E_tr = e^{tau A})."""
    n = 16
    h = 1.0 / n
    P = I.density_advection(n=n, u=0.5, v=0.0, p=0.1, amp=0.2, dt=h)  # u dt / h = 1/2
    st, fl = orc.step(P.state, P.grid.h, P.gamma, P.dt, variant)
    assert fl == 0
    old, new = P.state, st
    for base in (4, 8, 12):
        for k in (1, 2, 3):
            assert np.max(np.abs(new[base + k] - old[base + k])) < 1e-14
    wc, _ = orc.center_recovery(old, P.gamma)
    roll = lambda a: np.roll(a, 1, axis=1)  # value at i-1
    tol = 1e-13
    assert np.max(np.abs(new[4] - roll(old[12]))) < tol    # V(i,j) <- E_h(i-1,j)
    assert np.max(np.abs(new[8] - roll(wc[0]))) < tol      # E_v(i,j) <- centre(i-1,j)
    assert np.max(np.abs(new[12] - old[4])) < tol          # E_h(i,j) <- V(i,j)


def test_rb_equals_tai_when_increments_vanish(orc):
    P = I.density_advection(n=12, u=0.3, v=-0.2, p=1.0, amp=0.1)
    a, _ = orc.step(P.state, P.grid.h, P.gamma, P.dt, orc.TAI)
    b, _ = orc.step(P.state, P.grid.h, P.gamma, P.dt, orc.RB)
    assert np.max(np.abs(a - b)) < 1e-14


def _packet_point_error(orc, n, nu, variant, T=None):
    P = I.wave_packet(n, nu=nu, eps=EPS)
    if T is None:
        dt, ns = P.dt, 1
    else:
        ns = int(round(T / P.dt))
        dt = T / ns
    st, fl = orc.run(P.state, P.grid.h, P.gamma, dt, ns, variant)
    assert fl == 0
    ex = I.build_state(P.grid, lambda x, y: I.packet_prim(x, y, dt * ns, EPS))
    return np.max(np.abs(st[4:] - ex[4:])) / EPS


def test_packet_one_step_orders(orc):
    """One step of the point update on the mixed linearized packet: RB-TAI's defect
    is O(h^3), the additive RB's O(h^2) (Sec. 4.2 analysis; Fig. of one-step errors)."""
    slopes = {}
    for variant in (orc.TAI, orc.RB):
        e = [_packet_point_error(orc, n, 0.25, variant) for n in (16, 32, 64)]
        slopes[variant] = np.log2(e[1] / e[2])
    assert slopes[orc.TAI] > 2.8, slopes
    assert 1.8 < slopes[orc.RB] < 2.3, slopes


@pytest.mark.slow
def test_packet_repeated_step_orders(orc):
    """Fixed final time T = 1/4: RB-TAI converges at ~3rd order (nu = 0.25), RB at
    a lower order (nu = 0.15, below its stability limit 0.195185)."""
    e_tai = [_packet_point_error(orc, n, 0.25, orc.TAI, T=0.25) for n in (16, 32, 64)]
    e_rb = [_packet_point_error(orc, n, 0.15, orc.RB, T=0.25) for n in (16, 32, 64)]
    s_tai = np.log2(e_tai[1] / e_tai[2])
    s_rb = np.log2(e_rb[1] / e_rb[2])
    assert s_tai > 2.75, (e_tai, s_tai)
    assert s_rb < 2.5, (e_rb, s_rb)
    assert e_tai[2] < e_rb[2]


def test_vortex_converges_to_translated_exact(orc):
    """Isentropic vortex (Sec. 6.2) against the exact translate after t ~ 0.5:
    average-density error falls at least at second order, point error too."""
    errs = []
    for n in (16, 32):
        P = I.vortex(n=n, cfl=0.4)
        T = 0.5
        ns = int(np.ceil(T / P.dt))
        st, fl = orc.run(P.state, P.grid.h, P.gamma, T / ns, ns)
        assert fl == 0
        ex = I.vortex_exact(P.grid, T)
        errs.append(np.max(np.abs(st[0] - ex[0])))
    assert np.log2(errs[0] / errs[1]) > 2.3, errs


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


def test_radial_pulse_keeps_grid_symmetry(orc):
    P = I.pulse(n=16, amp=0.1, width2=0.1)
    st, fl = orc.run(P.state, P.grid.h, P.gamma, P.dt, 6)
    assert fl == 0
    assert np.max(np.abs(_mirror_x(P.state) - P.state)) < 1e-14
    assert np.max(np.abs(_mirror_x(st) - st)) < 1e-13
    assert np.max(np.abs(_swap_xy(st) - st)) < 1e-13
    assert np.max(np.abs(st[5])) > 1e-4  # the pulse has started to move


def test_centre_recovery_inverts_simpson(orc):
    """Averages built by the tensor Simpson rule from nodal conservative values and a
    chosen centre are inverted back to that centre (Eq. center-node)."""
    rng = np.random.default_rng(9)
    nx, ny, g = 6, 5, 1.4
    st = np.empty((16, ny, nx))
    for base in (4, 8, 12):
        st[base] = 1 + 0.2 * rng.random((ny, nx))
        st[base + 1] = rng.normal(size=(ny, nx))
        st[base + 2] = rng.normal(size=(ny, nx))
        st[base + 3] = 1 + 0.2 * rng.random((ny, nx))
    wc = np.stack([1 + 0.2 * rng.random((ny, nx)), rng.normal(size=(ny, nx)),
                   rng.normal(size=(ny, nx)), 1 + 0.2 * rng.random((ny, nx))])
    cons = lambda w: np.stack([w[0], w[0] * w[1], w[0] * w[2],
                               w[3] / (g - 1) + 0.5 * w[0] * (w[1] ** 2 + w[2] ** 2)])
    sh = lambda a, di, dj: np.roll(np.roll(a, -di, axis=-1), -dj, axis=-2)
    UV, UEv, UEh = cons(st[4:8]), cons(st[8:12]), cons(st[12:16])
    corners = UV + sh(UV, 1, 0) + sh(UV, 0, 1) + sh(UV, 1, 1)
    edges = UEh + sh(UEh, 0, 1) + UEv + sh(UEv, 1, 0)
    st[0:4] = corners / 36 + edges / 9 + 4 * cons(wc) / 9
    got, fl = orc.center_recovery(st, g)
    assert fl == 0
    assert np.max(np.abs(got - wc)) < 1e-12


def test_reconstruction_interpolates_q2_polynomials(orc):
    """R_h reproduces a Q2 polynomial inside a cell from its nine nodal values."""
    rng = np.random.default_rng(2)
    c = rng.normal(size=(4, 3, 3)) * 0.1
    c[0, 0, 0] = c[3, 0, 0] = 1.0
    poly = lambda k, x, y: np.polynomial.polynomial.polyval2d(x, y, c[k])
    nx = ny = 4
    st = np.zeros((16, ny, nx))
    # only cell (1,1) matters: nodes at x in {1, 1.5, 2}, y in {1, 1.5, 2} (cell units)
    for base, (ox, oy) in ((4, (0, 0)), (8, (0, 0.5)), (12, (0.5, 0))):
        for k in range(4):
            for j in range(ny):
                for i in range(nx):
                    st[base + k, j, i] = poly(k, (i + ox) / 4, (j + oy) / 4)
    wcen = [poly(k, 1.5 / 4, 1.5 / 4) for k in range(4)]
    g = 1.4
    cons = lambda w: np.array([w[0], w[0] * w[1], w[0] * w[2],
                               w[3] / (g - 1) + 0.5 * w[0] * (w[1] ** 2 + w[2] ** 2)])
    nodes = [(1, 1), (2, 1), (1, 2), (2, 2)]
    corners = sum(cons(st[4:8, j, i]) for i, j in nodes)
    edges = cons(st[12:16, 1, 1]) + cons(st[12:16, 2, 1]) + cons(st[8:12, 1, 1]) + cons(st[8:12, 1, 2])
    st[0:4, 1, 1] = corners / 36 + edges / 9 + 4 * cons(wcen) / 9
    st[0:4, :, :] += 0  # other cells unused
    st[0, :, :] = np.where(st[0] == 0, 1.0, st[0])
    st[3, :, :] = np.where(st[3] == 0, 2.5, st[3])
    for X, Y in rng.random((10, 2)) + 1.0:
        got = orc.recon_eval(st, g, X, Y)
        want = [poly(k, X / 4, Y / 4) for k in range(4)]
        assert np.max(np.abs(got - want)) < 1e-13


def test_flags_report_cfl_and_nonphysical_states(orc):
    P = I.random_smooth(8, 8, seed=1)
    _, fl = orc.step(P.state, P.grid.h, P.gamma, P.dt * 3.0)
    assert fl & orc.FLAG_CFL
    bad = P.state.copy()
    bad[4 + 3, 2, 3] = -1.0
    _, fl = orc.step(bad, P.grid.h, P.gamma, P.dt)
    assert fl & orc.FLAG_NONPHYSICAL
