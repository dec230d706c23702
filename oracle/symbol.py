"""Linearised Fourier symbol of the fully discrete scheme (Sec. 5, Appendix D).

TEST INFRASTRUCTURE ONLY (pins of the oracle; see the package docstring of
``oracle``).  Builds, for a uniform background W0 = (rho0, u0, v0, p0) and a
wave vector (xi, eta) in radians per cell, the 16x16 amplification matrix G_m
of one step acting on the Fourier amplitudes q = (w_bar, w^V, w^Ev, w^Eh) of
the four families in primitive perturbation variables:

* centre row  C(zx, zy) = [9/4, -(1+zx)(1+zy)/16, -(1+zx)/4, -(1+zy)/4]
  (linearised Simpson inversion, Appendix D);
* the value of a lattice node as a row over the families, with the phase of
  its cell; the Q2 reconstruction row at a point (floor convention for the
  cell, Appendix D);
* acoustic maps A_K (frozen at the background, r = nu sigma), taken from the
  oracle's exact acoustic node operator, which is linear in the data and is
  probed on unit vectors; density from the acoustic closure;
* advection D_K = reconstruction row at X_K - sigma lambda (u0, v0);
* RB: P_K = A_K + D_K - S_K;  RB-TAI: P_K = D_K + I_h(A - S)(X_K - d);
* average row: B - lambda (zx - 1) A_x E_x - lambda (zy - 1) A_y E_y with the
  space-time Simpson edge rows E and the primitive flux Jacobians A_x, A_y.

Everything is vectorised over a batch of wave vectors.
"""
import numpy as np

from . import NODE_C, NODE_EH, NODE_EV, NODE_V, RB, TAI, sac_node

# wedge cells of each family relative to the node's owner cell, and the node's
# lattice parity offset (a, b): lattice (2i + a, 2j + b)
_FAM = {
    NODE_V: ((0, 0), [(0, 0), (-1, 0), (-1, -1), (0, -1)]),
    NODE_EV: ((0, 1), [(0, 0), (-1, 0)]),
    NODE_EH: ((1, 0), [(0, 0), (0, -1)]),
    NODE_C: ((1, 1), [(0, 0)]),
}


def _lag(s):
    return np.array([0.5 * s * (s - 1.0), 1.0 - s * s, 0.5 * s * (s + 1.0)])


class Symbol:
    def __init__(self, nu, rho0=1.0, u0=0.0, v0=0.0, p0=1.0, gamma=1.4, variant=TAI):
        self.nu, self.gamma, self.variant = nu, gamma, variant
        self.w0 = np.array([rho0, u0, v0, p0], dtype=float)
        self.c0 = np.sqrt(gamma * p0 / rho0)
        self.Z0 = rho0 * self.c0
        self.lam = nu / self.c0  # dt / h
        # linear acoustic node maps for sigma = 1/2 and 1: coef[fam][s] with
        # shape (nwedge, 3 fields (p,u,v), 3, 3, 3 outputs (p,u,v))
        self.coef = {}
        for fam, (_, cells) in _FAM.items():
            for s, sig in enumerate((0.5, 1.0)):
                nw = len(cells)
                c = np.zeros((nw, 3, 3, 3, 3))
                for k in range(nw):
                    for f in range(3):
                        for ix in range(3):
                            for iy in range(3):
                                e = np.zeros((nw, 3, 3, 3))
                                e[k, f, ix, iy] = 1.0
                                c[k, f, ix, iy] = sac_node(fam, e, nu * sig, self.Z0)
                self.coef[(fam, s)] = c
        r, u, v, p = self.w0
        # primitive flux Jacobians A = M^{-1} dF/dW, M = dU/dW
        M = np.array([[1, 0, 0, 0], [u, r, 0, 0], [v, 0, r, 0],
                      [0.5 * (u * u + v * v), r * u, r * v, 1 / (gamma - 1)]])
        g1 = gamma / (gamma - 1)
        dF = np.array([[u, r, 0, 0], [u * u, 2 * r * u, 0, 1], [u * v, r * v, r * u, 0],
                       [0.5 * u * (u * u + v * v), g1 * p + 0.5 * r * (u * u + v * v) + r * u * u,
                        r * u * v, g1 * u]])
        dG = np.array([[v, 0, r, 0], [u * v, r * v, r * u, 0], [v * v, 0, 2 * r * v, 1],
                       [0.5 * v * (u * u + v * v), r * u * v,
                        g1 * p + 0.5 * r * (u * u + v * v) + r * v * v, g1 * v]])
        Mi = np.linalg.inv(M)
        self.Ax = Mi @ dF
        self.Ay = Mi @ dG

    # ---- rows over the four families (scalar), batch of wave vectors ------------
    def _cent(self, zx, zy):
        return np.stack([np.full_like(zx, 2.25), -(1 + zx) * (1 + zy) / 16, -(1 + zx) / 4,
                         -(1 + zy) / 4], axis=-1)

    def node_row(self, I, J, zx, zy):
        """Scalar value of lattice node (I, J) as a row over (avg, V, Ev, Eh)."""
        a, b = I & 1, J & 1
        ph = zx ** ((I - a) // 2) * zy ** ((J - b) // 2)
        if a == 0 and b == 0:
            e = np.array([0, 1, 0, 0], dtype=complex)
        elif a == 0 and b == 1:
            e = np.array([0, 0, 1, 0], dtype=complex)
        elif a == 1 and b == 0:
            e = np.array([0, 0, 0, 1], dtype=complex)
        else:
            return ph[:, None] * self._cent(zx, zy)
        return ph[:, None] * e[None, :]

    def recon_row(self, x, y, zx, zy):
        """Scalar Q2 reconstruction at (x, y) in cell units (floor convention)."""
        r, s = int(np.floor(x)), int(np.floor(y))
        lx, ly = _lag(2 * (x - r) - 1), _lag(2 * (y - s) - 1)
        out = 0
        for a in range(3):
            for b in range(3):
                out = out + lx[a] * ly[b] * self.node_row(2 * r + a, 2 * s + b, zx, zy)
        return out

    @staticmethod
    def _kron(row):
        """(K, 4) scalar row -> (K, 4, 16) block acting component-wise."""
        K = row.shape[0]
        out = np.zeros((K, 4, 16), dtype=complex)
        for c in range(4):
            for f in range(4):
                out[:, c, 4 * f + c] = row[:, f]
        return out

    def acoustic(self, fam, I, J, s, zx, zy):
        """A_K (K, 4, 16): (rho, u, v, p) after the frozen acoustic evolution of
        duration sigma dt at lattice node (I, J) of family fam."""
        (a, b), cells = _FAM[fam]
        ci, cj = (I - a) // 2, (J - b) // 2
        coef = self.coef[(fam, s)]
        K = zx.shape[0]
        out = np.zeros((K, 4, 16), dtype=complex)
        comp = {0: 3, 1: 1, 2: 2}  # field p,u,v -> primitive component
        for k, (di, dj) in enumerate(cells):
            for ix in range(3):
                for iy in range(3):
                    row = self.node_row(2 * (ci + di) + ix, 2 * (cj + dj) + iy, zx, zy)
                    for f in range(3):
                        for o in range(3):
                            cval = coef[k, f, ix, iy, o]
                            if cval != 0.0:
                                out[:, comp[o], 4 * np.arange(4) + comp[f]] += cval * row
        # density closure: rho_ac = rho_K + (p_ac - p_K) / c0^2
        self_row = self._kron(self.node_row(I, J, zx, zy))
        out[:, 0, :] = self_row[:, 0, :] + (out[:, 3, :] - self_row[:, 3, :]) / self.c0 ** 2
        return out

    def point_map(self, fam, s, zx, zy):
        """P_K^sigma (K, 4, 16) of the point family fam (V, Ev, Eh) at sigma = 1/2, 1."""
        a, b = _FAM[fam][0]
        sig = 0.5 if s == 0 else 1.0
        d = sig * self.lam * self.w0[1:3]
        X, Y = 0.5 * a - d[0], 0.5 * b - d[1]
        D = self._kron(self.recon_row(X, Y, zx, zy))
        S = self._kron(self.node_row(a, b, zx, zy))
        if self.variant == RB:
            return self.acoustic(fam, a, b, s, zx, zy) + D - S
        # transported increments: interpolate (A - S) of the foot cell's nodes
        r, t = int(np.floor(X)), int(np.floor(Y))
        lx, ly = _lag(2 * (X - r) - 1), _lag(2 * (Y - t) - 1)
        inc = 0
        for ia in range(3):
            for ib in range(3):
                I, J = 2 * r + ia, 2 * t + ib
                nf = {(0, 0): NODE_V, (0, 1): NODE_EV, (1, 0): NODE_EH, (1, 1): NODE_C}[(I & 1, J & 1)]
                Dn = self.acoustic(nf, I, J, s, zx, zy) - self._kron(self.node_row(I, J, zx, zy))
                inc = inc + lx[ia] * ly[ib] * Dn
        return D + inc

    def matrix(self, xi, eta):
        """G_m for arrays of wave numbers (radians per cell): shape (K, 16, 16)."""
        xi = np.atleast_1d(np.asarray(xi, dtype=float))
        eta = np.atleast_1d(np.asarray(eta, dtype=float))
        zx, zy = np.exp(1j * xi), np.exp(1j * eta)
        K = zx.shape[0]
        P = {}
        for fam in (NODE_V, NODE_EV, NODE_EH):
            a, b = _FAM[fam][0]
            P[(fam, -1)] = self._kron(self.node_row(a, b, zx, zy))  # sigma = 0
            for s in (0, 1):
                P[(fam, s)] = self.point_map(fam, s, zx, zy)
        E = {}
        for s in (-1, 0, 1):
            E[("x", s)] = ((1 + zy)[:, None, None] * P[(NODE_V, s)] + 4 * P[(NODE_EV, s)]) / 6
            E[("y", s)] = ((1 + zx)[:, None, None] * P[(NODE_V, s)] + 4 * P[(NODE_EH, s)]) / 6
        Ex = (E[("x", -1)] + 4 * E[("x", 0)] + E[("x", 1)]) / 6
        Ey = (E[("y", -1)] + 4 * E[("y", 0)] + E[("y", 1)]) / 6
        B = np.zeros((K, 4, 16), dtype=complex)
        B[:, :, 0:4] = np.eye(4)
        Gav = B - self.lam * (zx - 1)[:, None, None] * np.einsum("ij,kjl->kil", self.Ax, Ex) \
            - self.lam * (zy - 1)[:, None, None] * np.einsum("ij,kjl->kil", self.Ay, Ey)
        G = np.concatenate([Gav, P[(NODE_V, 1)], P[(NODE_EV, 1)], P[(NODE_EH, 1)]], axis=1)
        return G

    def spectral_radius(self, xi, eta):
        return np.max(np.abs(np.linalg.eigvals(self.matrix(xi, eta))), axis=-1)


def packet_background(mach=0.2, phi_deg=25.0):
    """The mixed-packet background of Sec. 4.2: rho0 = p0 = 1, |u0| = M at phi."""
    return dict(rho0=1.0, p0=1.0, u0=mach * np.cos(np.radians(phi_deg)),
                v0=mach * np.sin(np.radians(phi_deg)))
