"""Pins of the oracle's exact frozen acoustic operator S_ac (Sec. 3.1, Appendix D)
against results fixed independently of its own closed form:

* the stencils printed in Appendix B (vertical-edge node, both halves);
* the finite Taylor series exp(r L) of linear acoustics for polynomial data
  (full disk, and any node whose adjacent cells carry one common polynomial);
* 1D d'Alembert solutions for data varying in one direction only, with a kink
  at the node (quadrants and half planes);
* the 2D Poisson (spherical-mean) formula for the pressure, evaluated by
  numerical cubature wedge by wedge;
* rotation / reflection equivariance of the node operators.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "appendix_b_vertical_edge_stencils.txt")
RS = [0.05, 0.2, 0.37, 0.5]
V, EV, EH, C = 0, 1, 2, 3
NWEDGE = {V: 4, EV: 2, EH: 2, C: 1}
# position of the node inside each adjacent cell (cell units from its lower-left
# corner), in the oracle's wedge order (V: NE, NW, SW, SE; E_v: right, left;
# E_h: upper, lower; C: full).  This is the geometry of Sec. 3.1.
NODE_IN_CELL = {
    V: [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)],
    EV: [(0.0, 0.5), (1.0, 0.5)],
    EH: [(0.5, 0.0), (0.5, 1.0)],
    C: [(0.5, 0.5)],
}
WEDGE_ANGLES = {  # angular extent of each wedge, same order
    V: [(0, np.pi / 2), (np.pi / 2, np.pi), (np.pi, 1.5 * np.pi), (1.5 * np.pi, 2 * np.pi)],
    EV: [(-np.pi / 2, np.pi / 2), (np.pi / 2, 1.5 * np.pi)],
    EH: [(0, np.pi), (np.pi, 2 * np.pi)],
    C: [(0, 2 * np.pi)],
}


def load_golden():
    tab = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            side, blk, row, col, expr = line.split(maxsplit=4)
            tab[(side, blk, int(row), int(col))] = expr
    return tab


def ev(expr, nu):
    return float(eval(expr, {"__builtins__": {}}, {"nu": nu}))


def node_xy(fam, k):
    """Node offsets of the 3x3 Q2 nodes of wedge cell k, relative to the target node."""
    ox, oy = NODE_IN_CELL[fam][k]
    xs = np.array([0.0, 0.5, 1.0]) - ox
    ys = np.array([0.0, 0.5, 1.0]) - oy
    return xs, ys


def cells_from_fn(fam, fn):
    """(nwedge, 3 fields, 3, 3) nodal arrays of (p, u, v) from fn(k, X, Y) -> (p, u, v)."""
    out = np.zeros((NWEDGE[fam], 3, 3, 3))
    for k in range(NWEDGE[fam]):
        xs, ys = node_xy(fam, k)
        for ix in range(3):
            for iy in range(3):
                out[k, :, ix, iy] = fn(k, xs[ix], ys[iy])
    return out


# ---------------------------------------------------------------- App. B ----
@pytest.mark.parametrize("r", RS)
def test_vertical_edge_matches_appendix_b(orc, r):
    tab = load_golden()
    Z = 1.7
    side_k = {"R": 0, "L": 1}
    # (block, input field, output index, scale): outputs ordered (p, u, v)
    uses = [("uu", 1, 1, 1.0), ("uv", 2, 1, 1.0), ("uv", 1, 2, 1.0), ("up", 0, 1, 1.0 / Z),
            ("up", 1, 0, Z), ("vv", 2, 2, 1.0), ("vp", 0, 2, 1.0 / Z), ("vp", 2, 0, Z),
            ("pp", 0, 0, 1.0)]
    worst = 0.0
    for side, k in side_k.items():
        for blk, fin, oidx, scale in uses:
            for row in range(3):
                for col in range(3):
                    cells = np.zeros((2, 3, 3, 3))
                    cells[k, fin, row, col] = 1.0
                    got = orc.sac_node(EV, cells, r, Z)[oidx]
                    want = scale * ev(tab[(side, blk, row, col)], r)
                    worst = max(worst, abs(got - want))
    assert worst < 1e-13, worst


# ---------------------------------------------- Taylor series exp(rL) -------
def taylor_node(cp, cu, cv, r, Z):
    """exp(rL)(pi,u,v) at the origin for polynomial data, L = -(u_X+v_Y, pi_X, pi_Y);
    c*: 2D coefficient arrays [a][b] of X^a Y^b, pi = p / Z."""
    P = np.polynomial.polynomial
    pi, u, v = cp / Z, cu.copy(), cv.copy()
    out = np.zeros(3)
    fact = 1.0
    for k in range(0, 8):
        if k > 0:
            fact *= k
        out += r ** k / fact * np.array([pi[0, 0], u[0, 0], v[0, 0]])
        dux = P.polyder(u, axis=0)
        dvy = P.polyder(v, axis=1)
        dpx = P.polyder(pi, axis=0)
        dpy = P.polyder(pi, axis=1)
        npi = -(np.pad(dux, ((0, 1), (0, 0))) + np.pad(dvy, ((0, 0), (0, 1))))
        nu_ = -np.pad(dpx, ((0, 1), (0, 0)))
        nv_ = -np.pad(dpy, ((0, 0), (0, 1)))
        pi, u, v = npi, nu_, nv_
    return np.array([Z * out[0], out[1], out[2]])


def eval_poly(c, X, Y):
    return np.polynomial.polynomial.polyval2d(X, Y, c)


@pytest.mark.parametrize("fam", [C, V, EV, EH])
@pytest.mark.parametrize("r", RS)
def test_common_polynomial_matches_taylor(orc, fam, r):
    """Adjacent cells carrying one common Q2 polynomial: the wedges together cover
    the full disk, so the node value is the finite Taylor series exp(rL)."""
    rng = np.random.default_rng(int(100 * r) + fam)
    Z = 1.3
    cp, cu, cv = (rng.normal(size=(3, 3)) for _ in range(3))
    cells = cells_from_fn(fam, lambda k, X, Y: (eval_poly(cp, X, Y), eval_poly(cu, X, Y),
                                                eval_poly(cv, X, Y)))
    got = orc.sac_node(fam, cells, r, Z)
    want = taylor_node(cp, cu, cv, r, Z)
    assert np.max(np.abs(got - want)) < 1e-12 * max(1.0, np.max(np.abs(want)))


# ------------------------------------------------------- d'Alembert ---------
def dalembert(pi_minus, pi_plus, s_minus, s_plus, r):
    """1D linear acoustics along a line: w+ = pi + s moves in +, w- = pi - s moves in -.
    pi_minus/s_minus: data on the negative side, pi_plus/s_plus on the positive side."""
    wp = pi_minus(-r) + s_minus(-r)
    wm = pi_plus(r) - s_plus(r)
    return 0.5 * (wp + wm), 0.5 * (wp - wm)


@pytest.mark.parametrize("fam,direction", [(V, 0), (V, 1), (EV, 0), (EV, 1), (EH, 0), (EH, 1)])
@pytest.mark.parametrize("r", RS)
def test_one_dimensional_data_is_dalembert(orc, fam, direction, r):
    """Data depending on one coordinate only, with a kink at the node where the
    node lies on a cell boundary across that direction, evolves by the 1D
    d'Alembert formula; the transverse velocity stays zero."""
    rng = np.random.default_rng(7 + fam + 10 * direction)
    Z = 0.8
    a0p, a0s = rng.normal(size=2)
    cl = rng.normal(size=(2, 2))  # (pi, s) slope/curvature on the negative side
    cr = rng.normal(size=(2, 2))
    if (fam, direction) in ((EV, 1), (EH, 0)):
        cr = cl  # the node lies inside its cells along this direction: no kink there
    neg = [lambda t, f=f: (a0p, a0s)[f] + cl[f, 0] * t + cl[f, 1] * t * t for f in range(2)]
    pos = [lambda t, f=f: (a0p, a0s)[f] + cr[f, 0] * t + cr[f, 1] * t * t for f in range(2)]

    def fn(k, X, Y):
        t = X if direction == 0 else Y
        side = pos if t > 0 else neg
        pi, s = side[0](t), side[1](t)
        if direction == 0:
            return Z * pi, s, 0.0
        return Z * pi, 0.0, s

    cells = cells_from_fn(fam, fn)
    got = orc.sac_node(fam, cells, r, Z)
    pi, s = dalembert(neg[0], pos[0], neg[1], pos[1], r)
    want = (Z * pi, s, 0.0) if direction == 0 else (Z * pi, 0.0, s)
    assert np.max(np.abs(got - np.array(want))) < 1e-13


# ---------------------------------------------- Poisson formula, cubature --
def wedge_moment_cubature(a, b, t0, t1, n=64):
    """(1/2pi) int_wedge int_0^1 rho^{a+b} cos^a sin^b rho d rho d theta / sqrt(1-rho^2)
    by Gauss-Legendre cubature in theta and in phi (rho = sin phi)."""
    x, w = np.polynomial.legendre.leggauss(n)
    th = 0.5 * (t1 - t0) * (x + 1) + t0
    ang = 0.5 * (t1 - t0) * np.sum(w * np.cos(th) ** a * np.sin(th) ** b)
    ph = 0.25 * np.pi * (x + 1)
    rad = 0.25 * np.pi * np.sum(w * np.sin(ph) ** (a + b + 1))
    return ang * rad / (2 * np.pi)


def monomials_of_cell(values, xs, ys):
    """Monomial coefficients [a][b] of the Q2 interpolant of 3x3 nodal values by
    solving the 9x9 Vandermonde system."""
    A = np.array([[x ** a * y ** b for a in range(3) for b in range(3)] for x in xs for y in ys])
    rhs = np.array([values[ix, iy] for ix in range(3) for iy in range(3)])
    return np.linalg.solve(A, rhs).reshape(3, 3)


def lattice_cells(fam, rng, Z):
    """Random continuous piecewise-Q2 data: nodal values on the half-cell lattice
    shared by the adjacent cells."""
    lat = {}

    def val(X, Y):
        key = (round(2 * X), round(2 * Y))
        if key not in lat:
            lat[key] = rng.normal(size=3) * np.array([Z, 1.0, 1.0])
        return lat[key]

    return cells_from_fn(fam, lambda k, X, Y: val(X, Y))


@pytest.mark.parametrize("fam", [V, EV, EH, C])
@pytest.mark.parametrize("r", RS)
def test_pressure_matches_poisson_cubature(orc, fam, r):
    """pi(0,t) = d/dt [t M[pi0]] + t M[-c div u0] (2D Poisson formula for the
    wave equation pi_tt = c^2 Lap pi), with the disk means split over the wedges
    and computed by cubature; scaled units c = h = 1, t = r."""
    rng = np.random.default_rng(3 + fam + int(1000 * r))
    Z = 1.6
    cells = lattice_cells(fam, rng, Z)
    P = np.polynomial.polynomial
    total = 0.0
    for k, (t0, t1) in enumerate(WEDGE_ANGLES[fam]):
        xs, ys = node_xy(fam, k)
        cp = monomials_of_cell(cells[k, 0], xs, ys) / Z
        cu = monomials_of_cell(cells[k, 1], xs, ys)
        cv = monomials_of_cell(cells[k, 2], xs, ys)
        div = np.zeros((3, 3))
        div[:2, :] += P.polyder(cu, axis=0)
        div[:, :2] += P.polyder(cv, axis=1)
        for a in range(3):
            for b in range(3):
                m = wedge_moment_cubature(a, b, t0, t1)
                q = a + b
                total += (q + 1) * r ** q * cp[a, b] * m
                total += -r ** (q + 1) * div[a, b] * m
    got = orc.sac_node(fam, cells, r, Z)[0]
    assert abs(got - Z * total) < 1e-12


# ------------------------------------------------------ equivariance --------
@pytest.mark.parametrize("r", RS)
def test_vertex_rotation_equivariance(orc, r):
    """Rotating the data by 90 degrees about a vertex rotates the result."""
    rng = np.random.default_rng(11)
    Z = 1.1
    lat = {}
    for X in range(-2, 3):
        for Y in range(-2, 3):
            lat[(X, Y)] = rng.normal(size=3)

    def data(rot):
        def fn(k, X, Y):
            key = (round(2 * X), round(2 * Y))
            if rot:
                src = (key[1], -key[0])  # value at R^{-1} x for a CCW rotation R
                p, u, v = lat[src]
                return p, -v, u
            return tuple(lat[key])
        return cells_from_fn(V, fn)

    a = orc.sac_node(V, data(False), r, Z)
    b = orc.sac_node(V, data(True), r, Z)
    assert np.max(np.abs(b - np.array([a[0], -a[2], a[1]]))) < 1e-13


@pytest.mark.parametrize("r", RS)
def test_edge_families_related_by_diagonal_reflection(orc, r):
    """Reflecting x <-> y (and u <-> v) maps an E_v node problem to an E_h one."""
    rng = np.random.default_rng(5)
    lat = {}

    def val(key):
        if key not in lat:
            lat[key] = rng.normal(size=3)
        return lat[key]

    ev_cells = cells_from_fn(EV, lambda k, X, Y: val((round(2 * X), round(2 * Y))))
    def eh_fn(k, X, Y):
        p, u, v = val((round(2 * Y), round(2 * X)))
        return p, v, u
    eh_cells = cells_from_fn(EH, eh_fn)
    a = orc.sac_node(EV, ev_cells, r, 0.9)
    b = orc.sac_node(EH, eh_cells, r, 0.9)
    assert np.max(np.abs(b - np.array([a[0], a[2], a[1]]))) < 1e-13


def test_constant_state_is_fixed(orc):
    for fam in (V, EV, EH, C):
        cells = np.zeros((NWEDGE[fam], 3, 3, 3))
        cells[:, 0] = 2.0
        cells[:, 1] = -0.3
        cells[:, 2] = 0.7
        out = orc.sac_node(fam, cells, 0.45, 1.9)
        assert np.allclose(out, [2.0, -0.3, 0.7], atol=1e-14, rtol=0)
