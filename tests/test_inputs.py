"""The seeded workload recipes sample what the benchmark configurations state
(point values at their nodes, averages by quadrature, time step from the CFL
number), checked on small copies of each workload.  No method arithmetic: the
recipes only sample analytic initial data."""
import numpy as np

from workloads import inputs as I

G = 1.4


def _nodes(g, ox, oy):
    x = g.x0 + g.h * (np.arange(g.nx) + ox)
    y = g.y0 + g.h * (np.arange(g.ny) + oy)
    return np.meshgrid(x, y)


def _cfl(P, cfl):
    return I.dt_from_cfl(P.state, P.grid, cfl, P.gamma) == P.dt


def test_shear_layer():
    P = I.shear(n=64)
    g = P.grid
    assert (g.x0, g.y0, g.nx * g.h) == (0.0, 0.0, 1.0)
    for base, (ox, oy) in ((4, (0, 0)), (8, (0, 0.5)), (12, (0.5, 0))):
        X, Y = _nodes(g, ox, oy)
        u = np.where(Y <= 0.5, np.tanh(80 * (Y - 0.25)), np.tanh(80 * (0.75 - Y)))
        assert np.allclose(P.state[base], 1.0)
        assert np.allclose(P.state[base + 1], u, atol=1e-15)
        assert np.allclose(P.state[base + 2], 0.05 * np.sin(2 * np.pi * X), atol=1e-15)
        assert np.allclose(P.state[base + 3], 1 / (G * 0.01))  # Mach 0.1: c = 10
    assert np.allclose(P.state[0], 1.0, atol=1e-14)  # mass average of rho = 1
    # dt from CFL 0.4 over max(|u| + c) at the point nodes
    c = np.sqrt(G * (1 / (G * 0.01)))
    speed = np.max(np.hypot(P.state[[5, 9, 13]], P.state[[6, 10, 14]])) + c
    assert abs(P.dt - 0.4 * g.h / speed) < 1e-15 and _cfl(P, 0.4)


def test_gaussian_pulse():
    P = I.pulse(n=64)
    g = P.grid
    assert (g.x0, g.y0, g.nx * g.h) == (-1.0, -1.0, 2.0)
    X, Y = _nodes(g, 0, 0)
    rho = 1 + 0.1 * np.exp(-(X ** 2 + Y ** 2) / 0.01)
    assert np.allclose(P.state[4], rho, atol=1e-15)
    assert np.all(P.state[[5, 6, 9, 10, 13, 14]] == 0.0)
    assert np.allclose(P.state[7], rho ** G, atol=1e-15)
    assert _cfl(P, 0.4) and P.n_steps == 400


def test_kelvin_helmholtz():
    P = I.kelvin_helmholtz(n=32)
    g = P.grid
    assert (g.x0, g.y0, g.nx * g.h) == (0.0, 0.0, 1.0)
    for base, (ox, oy) in ((4, (0, 0)), (8, (0, 0.5)), (12, (0.5, 0))):
        X, Y = _nodes(g, ox, oy)
        inside = np.abs(Y - 0.5) < 0.25
        assert np.array_equal(P.state[base], np.where(inside, 2.0, 1.0))
        assert np.array_equal(P.state[base + 1], np.where(inside, 0.5, -0.5))
        assert np.allclose(P.state[base + 2], 0.01 * np.sin(4 * np.pi * X), atol=1e-15)
        assert np.all(P.state[base + 3] == 2.5)
    assert _cfl(P, 0.4) and P.n_steps == 1000


def test_isentropic_vortex():
    P = I.vortex(n=32)
    g = P.grid
    assert (g.x0, g.y0, g.nx * g.h) == (-5.0, -5.0, 10.0)
    X, Y = _nodes(g, 0, 0)
    r2 = X ** 2 + Y ** 2
    beta = 5.0
    T = 1 - (G - 1) * beta ** 2 / (8 * G * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1 / (G - 1))
    du = -beta / (2 * np.pi) * np.exp((1 - r2) / 2) * Y
    dv = beta / (2 * np.pi) * np.exp((1 - r2) / 2) * X
    assert np.allclose(P.state[4], rho, atol=1e-14)
    assert np.allclose(P.state[5], 1 + du, atol=1e-14)
    assert np.allclose(P.state[6], 1 + dv, atol=1e-14)
    assert np.allclose(P.state[7], rho ** G, atol=1e-14)
    assert _cfl(P, 0.4) and P.n_steps == 100


def test_vortex_ensemble_is_seeded_and_in_range():
    a, b = I.ensemble(), I.ensemble()
    assert a == b and len(a) == 256
    assert {s["n"] for s in a} == {64, 128, 256, 512}
    for s in a:
        assert 3.0 <= s["beta"] <= 5.0
        assert -1.0 <= s["uinf"] <= 1.0 and -1.0 <= s["vinf"] <= 1.0
        assert s["cfl"] == 0.4 and s["n_steps"] == 200
    assert I.ensemble(seed=1) != a


def test_averages_are_gauss_quadrature_of_the_conserved_state():
    """For data polynomial in x and y of degree <= 11 per direction the 6-point
    Gauss-Legendre average is exact: rho = 1 + x y^2 on [0,1]^2 (averages of
    rho and of the energy with u = v = 0 and p = 1)."""
    g = I.grid_on(8, 8, 0.0, 1.0, 0.0, 1.0)
    st = I.build_state(g, lambda x, y: (1 + x * y * y, 0 * x, 0 * x, 1 + 0 * x), G)
    xa, xb = g.h * np.arange(8), g.h * (np.arange(8) + 1)
    mx = (xb ** 2 - xa ** 2) / 2 / g.h          # cell average of x
    my = (xb ** 3 - xa ** 3) / 3 / g.h          # cell average of y^2
    assert np.allclose(st[0], 1 + my[:, None] * mx[None, :], atol=1e-15)
    assert np.allclose(st[3], 1 / (G - 1), atol=1e-15)


def test_smooth_direction():
    g = I.grid_on(48, 40, 0.0, 1.2, 0.0, 1.0)
    d = I.smooth_direction(g, 3)
    assert d.shape == (16, 40, 48) and abs(np.max(np.abs(d)) - 1.0) < 1e-15
    assert np.array_equal(d, I.smooth_direction(g, 3))
    # smooth: neighbouring nodes differ by O(h), across the periodic seam too
    for p in range(16):
        assert np.max(np.abs(np.diff(d[p], axis=1, append=d[p][:, :1]))) < 20 * g.h
        assert np.max(np.abs(np.diff(d[p], axis=0, append=d[p][:1, :]))) < 20 * g.h
    # every node family samples the same function of a component: the vertex
    # and the horizontal-edge planes differ by half a cell only
    assert np.max(np.abs(d[4] - d[12])) < 10 * g.h
