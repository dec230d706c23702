"""Pins of the whole linearised step against the numbers Sec. 5 prints, through
the 16x16 Fourier symbol of oracle/symbol.py (Appendix D construction):

* the symbol is the linearisation of the oracle's step: it reproduces central
  differences of orc_step on a periodic 12x12 grid for Fourier-mode
  perturbations (TAI and RB);
* RB-TAI is spectrally stable up to the wedge-geometry ceiling nu = 1/2 on the
  packet background (Sec. 5.2: "0.500000 ... with no earlier spectral crossing");
* RB loses stability through a long-wave acoustic mode near 44.4 degrees at
  nu_crit close to the printed 0.195185 (Sec. 5.2); the crossing is computed
  with the smallest wave number kappa = 0.02, where |g| - 1 is resolved in FP64;
* RB-TAI's sampled powers through 1000 steps stay bounded near the printed
  maximum norm 3.87 at nu = 0.25 (Sec. 5.2);
* the one-step pressure gain of the right-running acoustic branch at the
  vertical-edge midpoint (Sec. 5.3, Eq. pressure-response): its largest
  distance from the exact gain over all directions at kappa = 1 equals the
  four printed values for nu = 0.2 ... 0.5 to their printed digits
  (tests/golden/sec5_3_tai_pressure_gain_maxima.txt).
"""
import numpy as np
import pytest

from workloads import inputs as I  # noqa: F401  (path set-up)


@pytest.fixture(scope="module")
def sym(orc):
    from oracle import symbol
    return symbol


@pytest.mark.parametrize("variant", [0, 1])
def test_symbol_is_the_linearised_oracle_step(orc, sym, variant):
    gamma, nu, Mc = 1.4, 0.25, 12
    S = sym.Symbol(nu, gamma=gamma, variant=variant, **sym.packet_background())
    h = 1.0 / Mc
    dt = nu * h / S.c0
    r, u, v, p = S.w0
    U0 = np.array([r, r * u, r * v, p / (gamma - 1) + 0.5 * r * (u * u + v * v)])
    Mm = np.array([[1, 0, 0, 0], [u, r, 0, 0], [v, 0, r, 0],
                   [0.5 * (u * u + v * v), r * u, r * v, 1 / (gamma - 1)]])
    x0 = np.empty((16, Mc, Mc))
    x0[0:4] = U0[:, None, None]
    for b in (4, 8, 12):
        x0[b:b + 4] = S.w0[:, None, None]
    rng = np.random.default_rng(variant)
    jj, ii = np.meshgrid(np.arange(Mc), np.arange(Mc), indexing="ij")
    worst = 0.0
    for m, n in ((1, 0), (2, 3), (5, 1), (3, 3), (6, 6)):
        xi, eta = 2 * np.pi * m / Mc, 2 * np.pi * n / Mc
        q = rng.normal(size=16) + 1j * rng.normal(size=16)
        Gq = S.matrix([xi], [eta])[0] @ q
        ph = np.exp(1j * (xi * ii + eta * jj))
        for part in (np.real, np.imag):
            d = np.empty_like(x0)
            d[0:4] = np.einsum("ij,jkl->ikl", Mm, part(q[0:4, None, None] * ph))
            for f in range(3):
                d[4 + 4 * f:8 + 4 * f] = part(q[4 + 4 * f:8 + 4 * f, None, None] * ph)
            eps = 1e-6
            yp, _ = orc.step(x0 + eps * d, h, gamma, dt, variant)
            ym, _ = orc.step(x0 - eps * d, h, gamma, dt, variant)
            dy = (yp - ym) / (2 * eps)
            dy[0:4] = np.einsum("ij,jkl->ikl", np.linalg.inv(Mm), dy[0:4])
            want = part(Gq[:, None, None] * ph)
            worst = max(worst, np.max(np.abs(dy - want)) / np.max(np.abs(want)))
    assert worst < 1e-8, worst


def _max_radius(S, kappas, n_theta=72):
    th = np.linspace(0, 2 * np.pi, n_theta + 1)[:-1]
    K, T = np.meshgrid(kappas, th)
    return float(np.max(S.spectral_radius((K * np.cos(T)).ravel(), (K * np.sin(T)).ravel())))


@pytest.mark.parametrize("nu", [0.1, 0.25, 0.4, 0.5])
def test_tai_is_stable_up_to_one_half(orc, sym, nu):
    S = sym.Symbol(nu, variant=orc.TAI, **sym.packet_background())
    assert _max_radius(S, np.linspace(0.02, np.pi, 40)) <= 1.0 + 1e-10


def _rb_long_wave(S, kappa):
    """max over directions of |g| - 1 at wave number kappa, and its direction (deg)."""
    g = lambda t: S.spectral_radius([kappa * np.cos(t)], [kappa * np.sin(t)])[0] - 1.0
    ths = np.radians(np.linspace(38.0, 52.0, 57))
    vals = [g(t) for t in ths]
    i = int(np.argmax(vals))
    lo, hi = ths[max(i - 1, 0)], ths[min(i + 1, len(ths) - 1)]
    for _ in range(40):
        m1, m2 = lo + 0.382 * (hi - lo), lo + 0.618 * (hi - lo)
        if g(m1) > g(m2):
            hi = m2
        else:
            lo = m1
    t = 0.5 * (lo + hi)
    return g(t), np.degrees(t)


def test_rb_critical_cfl_and_direction(orc, sym):
    bg = sym.packet_background()
    # stable below, unstable above, through long waves
    assert _max_radius(sym.Symbol(0.19, variant=orc.RB, **bg), np.linspace(0.02, np.pi, 30)) \
        <= 1.0 + 1e-12
    assert _rb_long_wave(sym.Symbol(0.20, variant=orc.RB, **bg), 0.02)[0] > 0
    lo, hi = 0.19, 0.20
    for _ in range(16):
        mid = 0.5 * (lo + hi)
        if _rb_long_wave(sym.Symbol(mid, variant=orc.RB, **bg), 0.02)[0] > 0:
            hi = mid
        else:
            lo = mid
    nu_c = 0.5 * (lo + hi)
    theta = _rb_long_wave(sym.Symbol(nu_c, variant=orc.RB, **bg), 0.02)[1]
    print("RB nu_crit %.6f at %.3f deg (printed 0.195185 at 44.427 deg)" % (nu_c, theta))
    assert abs(nu_c - 0.195185) < 1e-4, nu_c
    assert abs(theta - 44.427) < 0.5, theta


def test_tai_power_norms_stay_bounded(orc, sym):
    S = sym.Symbol(0.25, variant=orc.TAI, **sym.packet_background())
    th = np.linspace(0, 2 * np.pi, 37)[:-1]
    K, T = np.meshgrid(np.linspace(0.03, 0.3, 10), th)
    G = S.matrix((K * np.cos(T)).ravel(), (K * np.sin(T)).ravel())
    P = G.copy()
    best = 0.0
    for n in range(1, 1001):
        if n > 1:
            P = np.einsum("kij,kjl->kil", G, P)
        if n % 25 == 0:
            best = max(best, float(np.max(np.linalg.norm(P, ord=2, axis=(1, 2)))))
    print("RB-TAI max ||G^n||, n <= 1000:", best, "(printed 3.87)")
    assert 3.7 < best < 4.0, best


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                    "sec5_3_tai_pressure_gain_maxima.txt")


def _exact_right_running(xi, eta, bg, gamma):
    """The exact right-running acoustic plane wave of unit pressure on the
    background, as the 16 Fourier amplitudes of the symbol: primitive
    perturbation (1/c^2, n/(rho0 c), 1), its cell average (the product of the
    two one-dimensional averages of the phase) and the node values of the
    vertex, vertical-edge and horizontal-edge families."""
    c = np.sqrt(gamma * bg["p0"] / bg["rho0"])
    kap = np.hypot(xi, eta)
    W = np.array([1 / c ** 2, xi / kap / (bg["rho0"] * c), eta / kap / (bg["rho0"] * c), 1.0],
                 dtype=complex)

    def mean_phase(z):
        return 1.0 if abs(z) < 1e-12 else (np.exp(1j * z) - 1) / (1j * z)

    return np.concatenate([W * mean_phase(xi) * mean_phase(eta), W,
                           W * np.exp(0.5j * eta), W * np.exp(0.5j * xi)])


def test_tai_pressure_gain_matches_printed_maxima(orc, sym):
    """Reading: the background is the packet background of Sec. 4.2 and the
    exact gain of the branch on it carries the background's advection as well
    as the acoustic phase nu kappa: exp(-i (nu kappa + (dt/h) u0 . (xi, eta)))."""
    gamma, kap = 1.4, 1.0
    bg = sym.packet_background()
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    th = np.linspace(0.0, 2 * np.pi, 1441)[:-1]
    xi, eta = kap * np.cos(th), kap * np.sin(th)
    for nu_s, printed_s in rows:
        nu, printed = float(nu_s), float(printed_s)
        S = sym.Symbol(nu, gamma=gamma, variant=orc.TAI, **bg)
        G = S.matrix(xi, eta)
        worst = 0.0
        for k in range(th.size):
            q = _exact_right_running(xi[k], eta[k], bg, gamma)
            g = (G[k] @ q)[11] / q[11]  # pressure at the vertical-edge midpoint
            g_ex = np.exp(-1j * (nu * kap + S.lam * (bg["u0"] * xi[k] + bg["v0"] * eta[k])))
            worst = max(worst, abs(g - g_ex))
        print("nu %.1f: max |g - g_ex| = %.4e (printed %.2e)" % (nu, worst, printed))
        assert abs(worst - printed) <= 5e-6, (nu, worst, printed)  # half a printed unit
