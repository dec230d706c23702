"""Python handle on the FP64 CPU oracle (``af_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously-correct
restatement of the paper's algorithm (Sec. 6.1) used to check the CUDA path.
Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  It shares
no code with the CUDA library and imports nothing from the product package.

State arrays are numpy float64 of shape (16, ny, nx) in the plane order
documented in ``af_oracle.h``: averages (rho, rho u, rho v, E), then
(rho, u, v, p) at vertices, x-edge midpoints (E_v) and y-edge midpoints (E_h).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "af_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TAI = 0
RB = 1
FC = 2  # foot-centred exact acoustic update (Appendix C)
FLAG_CFL = 1
FLAG_NONPHYSICAL = 2
FLAG_NONFINITE = 4
NODE_V, NODE_EV, NODE_EH, NODE_C = 0, 1, 2, 3
NINV = 12
INVARIANT_NAMES = [
    "mass", "mom_x", "mom_y", "energy", "entropy_simpson", "entropy_avg",
    "kinetic_energy", "max_wave_speed", "min_rho", "min_p", "vorticity_integral", "flags",
]

_lib = None


def build(force=False):
    """Compile liboracle.so with gcc (plain C11, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "af_oracle.h"))
    ):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd, cwd=_HERE)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i, d = ctypes.c_int, ctypes.c_double
        lib.orc_step.argtypes = [i, i, d, d, d, i, dp, dp]
        lib.orc_step.restype = i
        lib.orc_run.argtypes = [i, i, d, d, d, i, i, dp]
        lib.orc_run.restype = i
        lib.orc_center_recovery.argtypes = [i, i, d, dp, dp]
        lib.orc_center_recovery.restype = i
        lib.orc_acoustic_increments.argtypes = [i, i, d, d, d, i, dp, dp, dp]
        lib.orc_acoustic_increments.restype = i
        lib.orc_sac_node.argtypes = [i, dp, d, d, dp]
        lib.orc_sac_node.restype = None
        lib.orc_fc_node.argtypes = [i, dp, d, d, d, d, dp]
        lib.orc_fc_node.restype = None
        lib.orc_sac_block.argtypes = [i, i, i, dp]
        lib.orc_sac_block.restype = None
        lib.orc_recon_eval.argtypes = [i, i, dp, dp, d, d, dp]
        lib.orc_recon_eval.restype = None
        lib.orc_invariants.argtypes = [i, i, d, d, dp, dp]
        lib.orc_invariants.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.ndim == 3 and a.shape[0] == 16, a.shape
    return a


def step(state, h, gamma, dt, variant=TAI):
    """One step (Sec. 6.1).  Returns (new_state, flags)."""
    st = _state(state)
    out = np.empty_like(st)
    ny, nx = st.shape[1:]
    flags = _load().orc_step(nx, ny, h, gamma, dt, variant, _ptr(st), _ptr(out))
    return out, flags


def run(state, h, gamma, dt, n_steps, variant=TAI):
    """n_steps steps.  Returns (new_state, flags)."""
    st = _state(state).copy()
    ny, nx = st.shape[1:]
    flags = _load().orc_run(nx, ny, h, gamma, dt, variant, n_steps, _ptr(st))
    return st, flags


def center_recovery(state, gamma):
    """Recovered primitive centre values, shape (4, ny, nx) (Eq. center-node)."""
    st = _state(state)
    ny, nx = st.shape[1:]
    wc = np.empty((4, ny, nx))
    flags = _load().orc_center_recovery(nx, ny, gamma, _ptr(st), _ptr(wc))
    return wc, flags


def acoustic_increments(state, h, gamma, tau, family):
    """(du, dv, dp) at every node of a family for duration tau, shape (3, ny, nx)."""
    st = _state(state)
    ny, nx = st.shape[1:]
    wc, _ = center_recovery(st, gamma)
    d = np.empty((3, ny, nx))
    flags = _load().orc_acoustic_increments(nx, ny, h, gamma, tau, family, _ptr(st), _ptr(wc),
                                            _ptr(d))
    return d, flags


def sac_node(family, cells, r, Z):
    """Exact frozen acoustic operator at one node.  cells: (nwedge, 3, 3, 3) array of
    (p, u, v) nodal values [field][ix][iy] in the family's wedge order.
    Returns (p_ac, u_ac, v_ac)."""
    c = np.ascontiguousarray(cells, dtype=np.float64).reshape(-1)
    out = np.empty(3)
    _load().orc_sac_node(family, _ptr(c), r, Z, _ptr(out))
    return out


def fc_node(family, cells, fx, fy, r, Z):
    """Foot-centred exact frozen acoustic evolution (Appendix C) at the foot
    F = P + (fx, fy) h of a point of `family` (V, EV or EH); cells as for
    sac_node, r = c tau / h, Z = rho c.  Returns (p, u, v) at F."""
    c = np.ascontiguousarray(cells, dtype=np.float64).reshape(-1)
    out = np.empty(3)
    _load().orc_fc_node(family, _ptr(c), fx, fy, r, Z, _ptr(out))
    return out


def sac_block(wedge, a, b):
    """Appendix D block C^Theta_ab as a 3x3 array, (pi,u,v) x (pi,u,v)."""
    out = np.empty(9)
    _load().orc_sac_block(wedge, a, b, _ptr(out))
    return out.reshape(3, 3)


def recon_eval(state, gamma, X, Y):
    """R_h W at a point in cell units; returns (rho, u, v, p)."""
    st = _state(state)
    ny, nx = st.shape[1:]
    wc, _ = center_recovery(st, gamma)
    out = np.empty(4)
    _load().orc_recon_eval(nx, ny, _ptr(st), _ptr(wc), X, Y, _ptr(out))
    return out


def invariants(state, h, gamma):
    """FP64 diagnostics, array of NINV values named by INVARIANT_NAMES."""
    st = _state(state)
    ny, nx = st.shape[1:]
    out = np.empty(NINV)
    _load().orc_invariants(nx, ny, h, gamma, _ptr(st), _ptr(out))
    return out
