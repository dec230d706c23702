"""Seeded synthetic inputs: initial conditions, grids and time steps.

This module is the only code shared by the CUDA path's tests/benchmark and the
oracle's tests.  It holds none of the method's arithmetic: it samples the
analytic initial data of each workload at the point nodes and integrates
the conservative state over each cell by 6x6 Gauss-Legendre quadrature, the
initialisation the paper describes (Sec. 6: averages by quadrature, point
values sampled).  Everything is FP64 numpy.

State layout: float64 array of shape (16, ny, nx); planes 0-3 are the cell
averages (rho, rho u, rho v, E) of C_ij, planes 4-7, 8-11 and 12-15 are the
primitive values (rho, u, v, p) at the vertex (x_i, y_j), the x-edge midpoint
(x_i, y_{j+1/2}) and the y-edge midpoint (x_{i+1/2}, y_j) (Sec. 2, Fig. 1).
"""
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4


@dataclass(frozen=True)
class Grid:
    """Periodic Cartesian grid of nx*ny square cells of side h, origin (x0, y0)."""
    nx: int
    ny: int
    x0: float
    y0: float
    h: float


def grid_on(nx, ny, xlo, xhi, ylo, yhi):
    h = (xhi - xlo) / nx
    assert abs((yhi - ylo) / ny - h) < 1e-12 * max(1.0, abs(h)), "cells must be square"
    return Grid(nx, ny, float(xlo), float(ylo), float(h))


def _cons(w, gamma):
    rho, u, v, p = w
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def build_state(grid, prim_fn, gamma=GAMMA, nq=6):
    """Average of U(W(x, y)) over each cell by nq x nq Gauss-Legendre quadrature,
    and W sampled at the vertex, x-edge and y-edge nodes.  prim_fn(x, y) returns
    (rho, u, v, p) arrays broadcast to x's shape."""
    nx, ny, h = grid.nx, grid.ny, grid.h
    xi = grid.x0 + h * np.arange(nx)[None, :]
    yj = grid.y0 + h * np.arange(ny)[:, None]
    st = np.empty((16, ny, nx))
    gx, gw = np.polynomial.legendre.leggauss(nq)
    acc = np.zeros((4, ny, nx))
    for a in range(nq):
        for b in range(nq):
            x = xi + 0.5 * h * (gx[a] + 1.0)
            y = yj + 0.5 * h * (gx[b] + 1.0)
            w = [np.broadcast_to(c, (ny, nx)) for c in prim_fn(x, y)]
            acc += 0.25 * gw[a] * gw[b] * _cons(np.stack(w), gamma)
    st[0:4] = acc
    for base, (ox, oy) in ((4, (0.0, 0.0)), (8, (0.0, 0.5)), (12, (0.5, 0.0))):
        x = xi + ox * h
        y = yj + oy * h
        w = prim_fn(np.broadcast_to(x, (ny, nx)), np.broadcast_to(y, (ny, nx)))
        for k in range(4):
            st[base + k] = np.broadcast_to(w[k], (ny, nx))
    return st


def max_wave_speed(state, gamma=GAMMA):
    """max over the point nodes of sqrt(u^2+v^2) + c (the CFL denominator, Sec. 6)."""
    s = 0.0
    for base in (4, 8, 12):
        rho, u, v, p = state[base:base + 4]
        s = max(s, float(np.max(np.sqrt(u * u + v * v) + np.sqrt(gamma * p / rho))))
    return s


def dt_from_cfl(state, grid, cfl, gamma=GAMMA):
    """dt = CFL h / max(|u| + c), fixed for the run."""
    return cfl * grid.h / max_wave_speed(state, gamma)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    grid: Grid
    gamma: float
    state: np.ndarray
    dt: float
    n_steps: int


def vortex_prim(x, y, xc=0.0, yc=0.0, beta=5.0, uinf=1.0, vinf=1.0, gamma=GAMMA,
                period=None):
    """Isentropic vortex (Sec. 6.2 form): free stream rho = p = 1, (uinf, vinf)."""
    dx, dy = x - xc, y - yc
    if period is not None:
        dx = dx - period[0] * np.round(dx / period[0])
        dy = dy - period[1] * np.round(dy / period[1])
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2 * np.pi) * f * dy
    dv = beta / (2 * np.pi) * f * dx
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    return rho, uinf + du, vinf + dv, rho ** gamma


def vortex(n=32, cfl=0.4, n_steps=100, beta=5.0, uinf=1.0, vinf=1.0, xc=0.0, yc=0.0,
           gamma=GAMMA):
    """Periodic [-5,5]^2 isentropic vortex convected by (uinf, vinf)."""
    g = grid_on(n, n, -5.0, 5.0, -5.0, 5.0)
    fn = lambda x, y: vortex_prim(x, y, xc, yc, beta, uinf, vinf, gamma, period=(10.0, 10.0))
    st = build_state(g, fn, gamma)
    return Problem("vortex", g, gamma, st, dt_from_cfl(st, g, cfl, gamma), n_steps)


def vortex_exact(grid, t, beta=5.0, uinf=1.0, vinf=1.0, xc=0.0, yc=0.0, gamma=GAMMA):
    """The convected vortex at time t (exact solution = translated initial data)."""
    fn = lambda x, y: vortex_prim(x, y, xc + uinf * t, yc + vinf * t, beta, uinf, vinf, gamma,
                                  period=(grid.nx * grid.h, grid.ny * grid.h))
    return build_state(grid, fn, gamma)


def pulse(n=512, cfl=0.4, n_steps=400, amp=0.1, width2=0.01, gamma=GAMMA):
    """Gaussian pressure pulse at rest on periodic [-1,1]^2: rho = 1 + amp exp(-r^2/width2),
    p = rho^gamma."""
    g = grid_on(n, n, -1.0, 1.0, -1.0, 1.0)

    def fn(x, y):
        rho = 1.0 + amp * np.exp(-(x * x + y * y) / width2)
        z = np.zeros_like(rho)
        return rho, z, z, rho ** gamma

    st = build_state(g, fn, gamma)
    return Problem("pulse", g, gamma, st, dt_from_cfl(st, g, cfl, gamma), n_steps)


def shear(n=2048, cfl=0.4, n_steps=2000, mach=0.1, gamma=GAMMA):
    """Doubly periodic low-Mach shear layer on [0,1]^2: rho = 1, p = 1/(gamma M^2),
    u = tanh(80(y-1/4)) for y <= 1/2 else tanh(80(3/4-y)), v = 0.05 sin(2 pi x)."""
    g = grid_on(n, n, 0.0, 1.0, 0.0, 1.0)

    def fn(x, y):
        u = np.where(y <= 0.5, np.tanh(80.0 * (y - 0.25)), np.tanh(80.0 * (0.75 - y)))
        v = 0.05 * np.sin(2 * np.pi * x)
        one = np.ones_like(u + v)
        return one, u + 0 * v, v + 0 * u, one / (gamma * mach * mach)

    st = build_state(g, fn, gamma)
    return Problem("shear", g, gamma, st, dt_from_cfl(st, g, cfl, gamma), n_steps)


def kelvin_helmholtz(n=1024, cfl=0.4, n_steps=1000, gamma=GAMMA):
    """Compressible KH on periodic [0,1]^2: rho = 2, u = 0.5 for |y-1/2| < 1/4, else
    rho = 1, u = -0.5; p = 2.5; v = 0.01 sin(4 pi x)."""
    g = grid_on(n, n, 0.0, 1.0, 0.0, 1.0)

    def fn(x, y):
        inside = np.abs(y - 0.5) < 0.25
        rho = np.where(inside, 2.0, 1.0) + 0 * x
        u = np.where(inside, 0.5, -0.5) + 0 * x
        v = 0.01 * np.sin(4 * np.pi * x) + 0 * y
        return rho, u, v, 2.5 + 0 * rho

    st = build_state(g, fn, gamma)
    return Problem("kh", g, gamma, st, dt_from_cfl(st, g, cfl, gamma), n_steps)


# ---- linearized Euler Fourier wave packet (Sec. 4.2) ----------------------
PACKET_K = {"entropy": (1, 2), "shear": (2, 1), "acoustic+": (3, 2), "acoustic-": (2, 3)}


def packet_prim(x, y, t, eps=1e-6, mach=0.2, phi_deg=25.0, gamma=GAMMA, modes=None):
    """Exact linear solution of the mixed packet at time t on the unit square."""
    rho0, p0 = 1.0, 1.0
    u0, v0 = mach * np.cos(np.radians(phi_deg)), mach * np.sin(np.radians(phi_deg))
    c0 = np.sqrt(gamma * p0 / rho0)
    modes = modes or list(PACKET_K)
    rho = rho0 + 0 * x
    u = u0 + 0 * x
    v = v0 + 0 * x
    p = p0 + 0 * x
    for name in modes:
        kx, ky = 2 * np.pi * np.array(PACKET_K[name], dtype=float)
        K = np.hypot(kx, ky)
        w0 = u0 * kx + v0 * ky
        if name == "entropy":
            rho = rho + eps * np.cos(kx * x + ky * y - w0 * t)
        elif name == "shear":
            ph = np.cos(kx * x + ky * y - w0 * t)
            u = u - eps * (ky / K) * ph
            v = v + eps * (kx / K) * ph
        else:
            s = 1.0 if name == "acoustic+" else -1.0
            ph = np.cos(kx * x + ky * y - (w0 + s * c0 * K) * t)
            p = p + eps * ph
            rho = rho + eps / c0 ** 2 * ph
            u = u + s * eps / (rho0 * c0) * (kx / K) * ph
            v = v + s * eps / (rho0 * c0) * (ky / K) * ph
    return rho, u, v, p


def wave_packet(n=56, nu=0.25, eps=1e-6, gamma=GAMMA, modes=None, t=0.0):
    """Packet on periodic [0,1]^2; dt from the acoustic CFL nu = c0 dt / h."""
    g = grid_on(n, n, 0.0, 1.0, 0.0, 1.0)
    st = build_state(g, lambda x, y: packet_prim(x, y, t, eps, gamma=gamma, modes=modes), gamma)
    c0 = np.sqrt(gamma)
    return Problem("packet", g, gamma, st, nu * g.h / c0, 0)


# ---- seeded random smooth states (parity inputs) --------------------------
def random_smooth(nx, ny, seed=0, amp=0.05, n_modes=4, flow=(0.3, -0.2), cfl=0.4,
                  gamma=GAMMA, h=None):
    """Uniform state plus n_modes random periodic Fourier modes per primitive
    field with relative amplitude amp; periodic domain of nx*ny unit-ish cells."""
    rng = np.random.default_rng(seed)
    h = h if h is not None else 1.0 / max(nx, ny)
    g = Grid(nx, ny, 0.0, 0.0, h)
    Lx, Ly = nx * h, ny * h
    base = np.array([1.0, flow[0], flow[1], 1.0 / gamma])
    modes = []
    for k in range(4):
        for _ in range(n_modes):
            mx = int(rng.integers(-3, 4))
            my = int(rng.integers(-3, 4))
            a = amp * (rng.random() - 0.5) * 2
            ph = rng.random() * 2 * np.pi
            modes.append((k, mx, my, a, ph))

    def fn(x, y):
        w = [base[k] + 0 * x for k in range(4)]
        for k, mx, my, a, ph in modes:
            scale = 1.0 if k in (0, 3) else 0.5
            w[k] = w[k] + (abs(base[k]) if k in (0, 3) else scale) * a * np.cos(
                2 * np.pi * (mx * x / Lx + my * y / Ly) + ph)
        return tuple(w)

    st = build_state(g, fn, gamma)
    return Problem("random", g, gamma, st, dt_from_cfl(st, g, cfl, gamma), 0)


def smooth_direction(grid, seed, n_modes=3):
    """Seeded smooth direction in state space, scaled to max |d| = 1: for each of
    the four components k a sum of n_modes periodic Fourier modes phi_k (wave
    numbers in [-3, 3] per axis), sampled at the cell centres (planes k) and at
    the vertex, x-edge and y-edge nodes (planes 4 + k, 8 + k, 12 + k).  Used as
    a perturbation or a finite-difference direction; being smooth across the
    node families, it does not excite grid-scale modes."""
    rng = np.random.default_rng(seed)
    nx, ny, h = grid.nx, grid.ny, grid.h
    Lx, Ly = nx * h, ny * h
    terms = [[(int(rng.integers(-3, 4)), int(rng.integers(-3, 4)), rng.uniform(-1.0, 1.0),
               rng.uniform(0.0, 2 * np.pi)) for _ in range(n_modes)] for _ in range(4)]

    def sample(k, ox, oy):
        x = (grid.x0 + h * (np.arange(nx) + ox)) / Lx
        y = (grid.y0 + h * (np.arange(ny) + oy)) / Ly
        out = np.zeros((ny, nx))
        for mx, my, a, ph in terms[k]:
            # separable: cos(A + B) = Re(e^{iA} e^{iB})
            out += a * np.real(np.exp(2j * np.pi * my * y + 1j * ph)[:, None] *
                               np.exp(2j * np.pi * mx * x)[None, :])
        return out

    d = np.empty((16, ny, nx))
    for k in range(4):
        d[k] = sample(k, 0.5, 0.5)
    for base, (ox, oy) in ((4, (0.0, 0.0)), (8, (0.0, 0.5)), (12, (0.5, 0.0))):
        for k in range(4):
            d[base + k] = sample(k, ox, oy)
    m = np.max(np.abs(d))
    return d / m if m > 0 else d


def uniform(nx, ny, rho=1.0, u=0.3, v=-0.7, p=0.9, cfl=0.4, gamma=GAMMA, h=0.1):
    g = Grid(nx, ny, 0.0, 0.0, h)
    st = build_state(g, lambda x, y: (rho + 0 * x, u + 0 * x, v + 0 * x, p + 0 * x), gamma)
    return Problem("uniform", g, gamma, st, dt_from_cfl(st, g, cfl, gamma), 0)


def density_advection(n=16, u=0.5, v=0.0, p=1.0, amp=0.2, gamma=GAMMA, dt=None):
    """Constant p and velocity with a smooth density perturbation on [0,1]^2:
    the frozen acoustic and advective generators commute (Sec. 4.1)."""
    g = grid_on(n, n, 0.0, 1.0, 0.0, 1.0)

    def fn(x, y):
        rho = 1.0 + amp * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
        return rho, u + 0 * x, v + 0 * x, p + 0 * x

    st = build_state(g, fn, gamma)
    if dt is None:
        dt = dt_from_cfl(st, g, 0.4, gamma)
    return Problem("density_advection", g, gamma, st, dt, 0)


def ensemble(n_problems=256, seed=0, sizes=(64, 128, 256, 512), cfl=0.4, n_steps=200,
             gamma=GAMMA):
    """Seeded ensemble of isentropic vortices on [-5,5]^2 of uneven sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_problems):
        n = int(rng.choice(sizes))
        beta = float(rng.uniform(3.0, 5.0))
        uinf, vinf = (float(c) for c in rng.uniform(-1.0, 1.0, size=2))
        xc, yc = (float(c) for c in rng.uniform(-2.5, 2.5, size=2))
        out.append(dict(n=n, beta=beta, uinf=uinf, vinf=vinf, xc=xc, yc=yc, cfl=cfl,
                        n_steps=n_steps))
    return out


def ensemble_member(spec, gamma=GAMMA):
    return vortex(n=spec["n"], cfl=spec["cfl"], n_steps=spec["n_steps"], beta=spec["beta"],
                  uinf=spec["uinf"], vinf=spec["vinf"], xc=spec["xc"], yc=spec["yc"],
                  gamma=gamma)
