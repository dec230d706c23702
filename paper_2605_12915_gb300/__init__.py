"""GB300-native RB-TAI Active Flux step (2D Euler, periodic Cartesian grid).

Thin ctypes binding of the C ABI in ``include/af.h``; every step of the method
runs in the CUDA kernels of ``libaf.so``.  The binding only marshals
arguments: numpy arrays or torch tensors in, pointers and sizes out.  There is
no CPU fallback: if ``libaf.so`` is missing or cannot be loaded, every call
raises.

State arrays have shape (16, ny, nx) and dtype float64 (see ``inputs``):
averages (rho, rho u, rho v, E), then (rho, u, v, p) at vertices, x-edge
midpoints and y-edge midpoints.
"""
import ctypes
import os

from . import _build

AF_OK, AF_ERR_ARG, AF_ERR_CUDA, AF_ERR_ALLOC, AF_ERR_CFL, AF_ERR_NONPHYSICAL, \
    AF_ERR_NONFINITE, AF_ERR_STATE, AF_ERR_TIMEOUT, AF_ERR_BOUNDS = range(10)
AF_FP64, AF_FP32, AF_FP32_COMP = 0, 1, 2
AF_TAI, AF_RB, AF_FC = 0, 1, 2
AF_HOST, AF_DEVICE = 0, 1
AF_NINV = 12
AF_BATCH_GEOMS = 4
INVARIANT_NAMES = ["mass", "mom_x", "mom_y", "energy", "entropy_simpson", "entropy_avg",
                   "kinetic_energy", "max_wave_speed", "min_rho", "min_p",
                   "vorticity_integral", "flags"]
PRECISIONS = {"fp64": AF_FP64, "fp32": AF_FP32, "fp32_comp": AF_FP32_COMP}
VARIANTS = {"tai": AF_TAI, "rb": AF_RB, "fc": AF_FC}

LIB_PATH = _build.LIB


class AfGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("h", ctypes.c_double)]


class AfState(ctypes.Structure):
    _fields_ = [("avg", ctypes.c_void_p * 4), ("vtx", ctypes.c_void_p * 4),
                ("ev", ctypes.c_void_p * 4), ("eh", ctypes.c_void_p * 4)]


class AfError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, af_status_string(status), status))


_lib = None


def load():
    """Load libaf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libaf.so not built: run paper_2605_12915_gb300._build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        lib.af_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(AfGrid), d,
                                ctypes.POINTER(AfState), ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, vp]
        lib.af_init.restype = ctypes.c_int
        lib.af_step.argtypes = [vp, d, i32]
        lib.af_step.restype = ctypes.c_int
        lib.af_sync.argtypes = [vp]
        lib.af_sync.restype = ctypes.c_int
        lib.af_get_state.argtypes = [vp, ctypes.POINTER(AfState), ctypes.c_int]
        lib.af_get_state.restype = ctypes.c_int
        lib.af_set_state.argtypes = [vp, ctypes.POINTER(AfState), ctypes.c_int]
        lib.af_set_state.restype = ctypes.c_int
        lib.af_exchange_state.argtypes = [vp, ctypes.POINTER(AfState), ctypes.POINTER(AfState),
                                          ctypes.c_int]
        lib.af_exchange_state.restype = ctypes.c_int
        lib.af_exchange_state_async.argtypes = [vp, ctypes.POINTER(AfState),
                                                ctypes.POINTER(AfState)]
        lib.af_exchange_state_async.restype = ctypes.c_int
        lib.af_reduce_invariants.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.af_reduce_invariants.restype = ctypes.c_int
        lib.af_adjoint_step.argtypes = [vp, d, ctypes.POINTER(AfState), ctypes.POINTER(AfState),
                                        ctypes.c_int]
        lib.af_adjoint_step.restype = ctypes.c_int
        lib.af_batch_init.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(AfGrid), d,
                                      ctypes.POINTER(AfState), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, vp]
        lib.af_batch_init.restype = ctypes.c_int
        lib.af_batch_step.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
        lib.af_batch_step.restype = ctypes.c_int
        lib.af_batch_sync.argtypes = [vp]
        lib.af_batch_sync.restype = ctypes.c_int
        lib.af_batch_get_state.argtypes = [vp, i32, ctypes.POINTER(AfState), ctypes.c_int]
        lib.af_batch_get_state.restype = ctypes.c_int
        lib.af_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
        lib.af_batch_info.restype = ctypes.c_int
        lib.af_batch_destroy.argtypes = [vp]
        lib.af_batch_destroy.restype = None
        lib.af_destroy.argtypes = [vp]
        lib.af_destroy.restype = None
        lib.af_status_string.argtypes = [ctypes.c_int]
        lib.af_status_string.restype = ctypes.c_char_p
        _lib = lib
    return _lib


# ---- raw C-ABI functions, same names -----------------------------------------
def af_status_string(status):
    return load().af_status_string(int(status)).decode()


def _state_struct(base_ptr, n):
    """AfState whose 16 planes are consecutive blocks of n doubles from base_ptr."""
    s = AfState()
    for k in range(4):
        s.avg[k] = base_ptr + 8 * n * k
        s.vtx[k] = base_ptr + 8 * n * (4 + k)
        s.ev[k] = base_ptr + 8 * n * (8 + k)
        s.eh[k] = base_ptr + 8 * n * (12 + k)
    return s


def _array_ptr(arr):
    """(pointer, on_device) of a C-contiguous float64 (16, ny, nx) numpy array or
    torch tensor."""
    if hasattr(arr, "data_ptr"):  # torch tensor
        import torch
        assert arr.dtype == torch.float64 and arr.is_contiguous() and arr.dim() == 3 \
            and arr.shape[0] == 16, "state must be a contiguous float64 (16, ny, nx) tensor"
        return arr.data_ptr(), arr.is_cuda
    import numpy as np
    assert isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.flags["C_CONTIGUOUS"] \
        and arr.ndim == 3 and arr.shape[0] == 16, \
        "state must be a C-contiguous float64 (16, ny, nx) array"
    return arr.ctypes.data, False


def af_init(nx, ny, h, gamma, state, precision=AF_FP32_COMP, variant=AF_TAI, stream=None):
    """Returns an opaque handle (int).  state: (16, ny, nx) float64 numpy array or
    torch tensor (host or cuda).  stream: torch.cuda.Stream, raw handle or None."""
    ptr, dev = _array_ptr(state)
    assert state.shape[1] == ny and state.shape[2] == nx
    g = AfGrid(nx, ny, h)
    st = _state_struct(ptr, nx * ny)
    hnd = ctypes.c_void_p()
    s = getattr(stream, "cuda_stream", stream)
    rc = load().af_init(ctypes.byref(hnd), ctypes.byref(g), gamma, ctypes.byref(st),
                        AF_DEVICE if dev else AF_HOST, precision, variant,
                        ctypes.c_void_p(s) if s else None)
    if rc != AF_OK:
        raise AfError(rc, "af_init")
    return hnd.value


def af_step(handle, dt, n_steps=1):
    return load().af_step(ctypes.c_void_p(handle), float(dt), int(n_steps))


def af_sync(handle):
    return load().af_sync(ctypes.c_void_p(handle))


def af_get_state(handle, out):
    ptr, dev = _array_ptr(out)
    n = out.shape[1] * out.shape[2]
    st = _state_struct(ptr, n)
    return load().af_get_state(ctypes.c_void_p(handle), ctypes.byref(st),
                               AF_DEVICE if dev else AF_HOST)


def af_set_state(handle, state):
    ptr, dev = _array_ptr(state)
    n = state.shape[1] * state.shape[2]
    st = _state_struct(ptr, n)
    return load().af_set_state(ctypes.c_void_p(handle), ctypes.byref(st),
                               AF_DEVICE if dev else AF_HOST)


def af_exchange_state(handle, out, state):
    """out <- the current state, then the current state <- state (both host or
    both device arrays of shape (16, ny, nx), float64)."""
    pout, dout = _array_ptr(out)
    pin, din = _array_ptr(state)
    assert dout == din, "out and state must both be host or both be device arrays"
    n = state.shape[1] * state.shape[2]
    so, si = _state_struct(pout, n), _state_struct(pin, n)
    return load().af_exchange_state(ctypes.c_void_p(handle), ctypes.byref(so), ctypes.byref(si),
                                     AF_DEVICE if din else AF_HOST)


def af_exchange_state_async(handle, out, state):
    """Enqueued form of af_exchange_state for host arrays (16, ny, nx) float64:
    `out` may be read and `state` modified only after af_sync."""
    pout, dout = _array_ptr(out)
    pin, din = _array_ptr(state)
    assert not dout and not din, "af_exchange_state_async takes host arrays"
    n = state.shape[1] * state.shape[2]
    so, si = _state_struct(pout, n), _state_struct(pin, n)
    return load().af_exchange_state_async(ctypes.c_void_p(handle), ctypes.byref(so),
                                           ctypes.byref(si))


def af_reduce_invariants(handle, out):
    """out: float64 numpy array of AF_NINV values (host)."""
    import numpy as np
    assert isinstance(out, np.ndarray) and out.dtype == np.float64 and out.size >= AF_NINV
    return load().af_reduce_invariants(ctypes.c_void_p(handle),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def af_adjoint_step(handle, dt, lam_in, lam_out):
    """lam_out = (d state^{n+1}/d state^n)^T lam_in about the handle's current state.
    Both (16, ny, nx) float64, both on the host (numpy) or both on the device (torch)."""
    pin, din = _array_ptr(lam_in)
    pout, dout = _array_ptr(lam_out)
    assert din == dout, "lam_in and lam_out must both be host or both be device arrays"
    n = lam_in.shape[1] * lam_in.shape[2]
    si, so = _state_struct(pin, n), _state_struct(pout, n)
    return load().af_adjoint_step(ctypes.c_void_p(handle), float(dt), ctypes.byref(si),
                                  ctypes.byref(so), AF_DEVICE if din else AF_HOST)


def af_destroy(handle):
    if handle:
        load().af_destroy(ctypes.c_void_p(handle))


# ---- convenience wrapper ---------------------------------------------------
class Solver:
    """One grid on the current CUDA device.

    >>> s = Solver(grid, gamma, state, precision="fp32_comp")
    >>> s.step(dt, 100); s.state()  # numpy (16, ny, nx) float64
    """

    def __init__(self, grid, gamma, state, precision="fp32_comp", variant="tai", stream=None):
        self.nx, self.ny, self.h, self.gamma = grid.nx, grid.ny, grid.h, gamma
        self.handle = af_init(grid.nx, grid.ny, grid.h, gamma, state,
                              PRECISIONS.get(precision, precision),
                              VARIANTS.get(variant, variant), stream)

    def step(self, dt, n_steps=1):
        rc = af_step(self.handle, dt, n_steps)
        if rc != AF_OK:
            raise AfError(rc, "af_step")

    def sync(self):
        rc = af_sync(self.handle)
        if rc != AF_OK:
            raise AfError(rc, "af_sync")

    def state(self, out=None):
        import numpy as np
        if out is None:
            out = np.empty((16, self.ny, self.nx))
        rc = af_get_state(self.handle, out)
        if rc != AF_OK:
            raise AfError(rc, "af_get_state")
        return out

    def set_state(self, state):
        rc = af_set_state(self.handle, state)
        if rc != AF_OK:
            raise AfError(rc, "af_set_state")

    def exchange(self, out, state):
        """Hand the current state out into `out` and take `state` in (see
        af_exchange_state); returns out."""
        rc = af_exchange_state(self.handle, out, state)
        if rc != AF_OK:
            raise AfError(rc, "af_exchange_state")
        return out

    def exchange_async(self, out, state):
        """Enqueue handing the current state out into `out` and taking `state`
        in (see af_exchange_state_async): `out` holds the result and `state` may
        be reused once sync() has returned."""
        rc = af_exchange_state_async(self.handle, out, state)
        if rc != AF_OK:
            raise AfError(rc, "af_exchange_state_async")
        return out

    def invariants(self):
        import numpy as np
        out = np.zeros(AF_NINV)
        rc = af_reduce_invariants(self.handle, out)
        if rc != AF_OK:
            raise AfError(rc, "af_reduce_invariants")
        return out

    def adjoint(self, dt, lam_in, lam_out=None):
        """Adjoint of one step about the current state (see af_adjoint_step)."""
        if lam_out is None:
            if hasattr(lam_in, "data_ptr"):
                lam_out = lam_in.new_empty(lam_in.shape)
            else:
                import numpy as np
                lam_out = np.empty_like(lam_in)
        rc = af_adjoint_step(self.handle, dt, lam_in, lam_out)
        if rc != AF_OK:
            raise AfError(rc, "af_adjoint_step")
        return lam_out

    def close(self):
        if self.handle:
            af_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """An ensemble of independent grids stepped together (af_batch_*).

    problems: sequence of objects with .grid, .gamma, .state (numpy (16, ny, nx)
    float64 host arrays), as built by ``inputs``; all share gamma."""

    def __init__(self, problems, precision="fp32", variant="tai", stream=None):
        import numpy as np
        n = len(problems)
        self.n = n
        self._states = [np.ascontiguousarray(p.state, dtype=np.float64) for p in problems]
        grids = (AfGrid * n)()
        states = (AfState * n)()
        for k, p in enumerate(problems):
            grids[k] = AfGrid(p.grid.nx, p.grid.ny, p.grid.h)
            states[k] = _state_struct(self._states[k].ctypes.data, p.grid.nx * p.grid.ny)
        self.shapes = [(p.grid.ny, p.grid.nx) for p in problems]
        hnd = ctypes.c_void_p()
        s = getattr(stream, "cuda_stream", stream)
        rc = load().af_batch_init(ctypes.byref(hnd), n, grids, problems[0].gamma, states, AF_HOST,
                                  PRECISIONS.get(precision, precision),
                                  VARIANTS.get(variant, variant), ctypes.c_void_p(s) if s else None)
        if rc != AF_OK:
            raise AfError(rc, "af_batch_init")
        self.handle = hnd.value

    def step(self, dts, n_steps=1):
        arr = (ctypes.c_double * self.n)(*[float(x) for x in dts])
        rc = load().af_batch_step(ctypes.c_void_p(self.handle), arr, int(n_steps))
        if rc != AF_OK:
            raise AfError(rc, "af_batch_step")

    def sync(self):
        rc = load().af_batch_sync(ctypes.c_void_p(self.handle))
        if rc != AF_OK:
            raise AfError(rc, "af_batch_sync")

    def state(self, k):
        import numpy as np
        out = np.empty((16,) + self.shapes[k])
        st = _state_struct(out.ctypes.data, out.shape[1] * out.shape[2])
        rc = load().af_batch_get_state(ctypes.c_void_p(self.handle), int(k), ctypes.byref(st),
                                       AF_HOST)
        if rc != AF_OK:
            raise AfError(rc, "af_batch_get_state")
        return out

    def info(self):
        g = ctypes.c_int32()
        t = (ctypes.c_float * AF_BATCH_GEOMS)()
        load().af_batch_info(ctypes.c_void_p(self.handle), ctypes.byref(g), t)
        return g.value, list(t)

    def close(self):
        if getattr(self, "handle", None):
            load().af_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
