"""Host-side checks of the CUDA library (no GPU needed): it builds for sm_103a,
loads, and exports every entry point include/af.h declares; the committed
generated stencil header is what its generator writes; the generated stencil
tables, applied on the CPU, reproduce the oracle's acoustic operator; and the
generated transposed stencils of the adjoint, evaluated on the CPU, are the
exact transpose of those tables.
"""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "af.h")
CSRC = os.path.join(ROOT, "paper_2605_12915_gb300", "csrc")
STENCILS = os.path.join(CSRC, "af_stencils.cuh")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(af_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libaf():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2605_12915_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_entry_point(libaf):
    syms = declared_symbols()
    assert {"af_init", "af_step", "af_reduce_invariants", "af_destroy"} <= set(syms)
    missing = [s for s in syms if not hasattr(libaf, s)]
    assert not missing, missing


def test_status_strings(libaf):
    libaf.af_status_string.restype = ctypes.c_char_p
    for s in range(10):
        assert libaf.af_status_string(s) != b"unknown status"
    assert libaf.af_status_string(10) == b"unknown status"


_BAD_INIT = {
    "nx < 2": dict(nx=1),
    "ny < 2": dict(ny=0),
    "negative size": dict(nx=-8),
    "h = 0": dict(h=0.0),
    "h NaN": dict(h=float("nan")),
    "gamma = 1": dict(gamma=1.0),
    "gamma NaN": dict(gamma=float("nan")),
    "unknown precision": dict(prec=3),
    "unknown variant": dict(var=3),
    "foot-centred variant in FP32": dict(var=2, prec=1),
    "foot-centred variant in FP32 compensated": dict(var=2, prec=2),
    "unknown memory kind": dict(where=2),
    "null state plane": dict(null_plane=5),
    "more than 2^31 cells": dict(nx=65536, ny=32769),
}


@pytest.mark.parametrize("case", sorted(_BAD_INIT))
def test_init_rejects_bad_arguments_without_touching_the_gpu(libaf, case):
    """Every invalid argument is refused with AF_ERR_ARG before any CUDA call
    (this runs on a machine without a GPU) and no handle is returned."""
    from paper_2605_12915_gb300 import AfGrid, AfState, AF_ERR_ARG
    arg = dict(nx=16, ny=16, h=0.1, gamma=1.4, prec=0, var=0, where=0, null_plane=None)
    arg.update(_BAD_INIT[case])
    buf = (ctypes.c_double * 16)()
    st = AfState()
    for k, field in enumerate(("avg", "vtx", "ev", "eh")):
        for q in range(4):
            getattr(st, field)[q] = None if arg["null_plane"] == 4 * k + q else ctypes.addressof(buf)
    h = ctypes.c_void_p()
    g = AfGrid(arg["nx"], arg["ny"], arg["h"])
    rc = libaf.af_init(ctypes.byref(h), ctypes.byref(g), ctypes.c_double(arg["gamma"]),
                       ctypes.byref(st), arg["where"], arg["prec"], arg["var"], None)
    assert rc == AF_ERR_ARG and not h.value


def test_binding_constants_match_the_header():
    import paper_2605_12915_gb300 as af
    text = open(HEADER).read()
    assert int(re.search(r"#define AF_BATCH_GEOMS (\d+)", text).group(1)) == af.AF_BATCH_GEOMS
    assert int(re.search(r"AF_NINV = (\d+)", text).group(1)) == af.AF_NINV
    assert int(re.search(r"AF_ERR_TIMEOUT = (\d+)", text).group(1)) == af.AF_ERR_TIMEOUT
    assert int(re.search(r"AF_ERR_BOUNDS = (\d+)", text).group(1)) == af.AF_ERR_BOUNDS
    assert int(re.search(r"AF_FC = (\d+)", text).group(1)) == af.AF_FC


def test_calls_on_a_null_handle_are_refused(libaf):
    from paper_2605_12915_gb300 import AF_ERR_ARG
    libaf.af_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32]
    assert libaf.af_step(None, ctypes.c_double(0.1), 1) == AF_ERR_ARG
    libaf.af_sync.argtypes = [ctypes.c_void_p]
    assert libaf.af_sync(None) == AF_ERR_ARG
    libaf.af_exchange_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int]
    assert libaf.af_exchange_state(None, None, None, 0) == AF_ERR_ARG
    libaf.af_exchange_state_async.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert libaf.af_exchange_state_async(None, None, None) == AF_ERR_ARG
    libaf.af_destroy.argtypes = [ctypes.c_void_p]
    libaf.af_destroy(None)  # a no-op


@pytest.mark.slow
def test_committed_stencils_match_generator(tmp_path):
    pytest.importorskip("sympy")
    out = tmp_path / "af_stencils.cuh"
    subprocess.check_call(["python", os.path.join(CSRC, "gen_stencils.py"), str(out)],
                          stdout=subprocess.DEVNULL)
    assert out.read_text() == open(STENCILS).read()


# ---- apply the generated tables on the CPU ---------------------------------
def parse_stencils():
    """{family: [(a, b, combo, field, dst, o, q, value)]} from the generated code."""
    fams = {}
    fam = None
    orbit = None
    for line in open(STENCILS):
        m = re.match(r"__device__ __forceinline__ void af_sac_(\w+)\(", line)
        if m:
            fam = m.group(1)
            fams[fam] = []
        m = re.search(r"orbit \(\+-(\d+), \+-(\d+)\)", line)
        if m:
            orbit = (int(m.group(1)), int(m.group(2)))
        m = re.search(r"(Gp|Guv)\[(\d)\]\[(\d)\] = fma\(T\(([-0-9.e]+)\), (ee|eo|oe|oo)(p|u|v),",
                      line)
        if m:
            fams[fam].append((orbit[0], orbit[1], m.group(5), m.group(6), m.group(1),
                              int(m.group(2)), int(m.group(3)) + 1, float(m.group(4))))
    return fams


def apply_tables(entries, lat, K):
    """G[o][q] for lattice data lat[(dx, dy)] = (p, u, v) around node value K."""
    Gp = np.zeros((3, 5))
    Guv = np.zeros((3, 5))
    fidx = {"p": 0, "u": 1, "v": 2}
    for a, b, combo, f, dst, o, q, val in entries:
        k = fidx[f]
        members = {(sx * a, sy * b) for sx in (1, -1) for sy in (1, -1)}
        tot = 0.0
        for (dx, dy) in members:
            sx = 1 if dx >= 0 else -1
            sy = 1 if dy >= 0 else -1
            wx = sx if combo[0] == "o" else 1
            wy = sy if combo[1] == "o" else 1
            dev = lat[(dx, dy)][k] - (K[k] if combo == "ee" else 0.0)
            tot += wx * wy * dev
        (Gp if dst == "Gp" else Guv)[o, q] += val * tot
    return Gp, Guv


@pytest.mark.parametrize("fam_name,fam", [("V", 0), ("EV", 1), ("EH", 2), ("C", 3)])
def test_generated_tables_match_oracle_operator(orc, fam_name, fam):
    from test_oracle_acoustic import cells_from_fn
    tables = parse_stencils()[fam_name]
    rng = np.random.default_rng(21 + fam)
    lat = {}
    Z = 1.45

    def val(X, Y):
        key = (round(2 * X), round(2 * Y))
        if key not in lat:
            lat[key] = rng.normal(size=3)
        return lat[key]

    cells = cells_from_fn(fam, lambda k, X, Y: val(X, Y))
    K = lat[(0, 0)]
    Gp, Guv = apply_tables(tables, lat, K)
    for r in (0.1, 0.3, 0.5):
        want = orc.sac_node(fam, cells, r, Z)  # (p_ac, u_ac, v_ac)
        pw = np.array([r ** q for q in range(5)])
        dp = np.sum(pw * (Gp[0] + Z * Guv[0]))
        du = np.sum(pw * (Gp[1] / Z + Guv[1]))
        dv = np.sum(pw * (Gp[2] / Z + Guv[2]))
        got = np.array([K[0] + dp, K[1] + du, K[2] + dv])
        assert np.max(np.abs(got - want)) < 1e-12, (r, got, want)


def parse_adjoint(fam_name):
    """The generated transposed stencil af_sac_<fam>_adj as a Python function
    (lGp, lGuv) -> ({(dx, dy): [lp, lu, lv]}, [lpK, luK, lvK]), by evaluating
    its statements in order (S.pair(dx, dy, member values, mirror values)
    scatters to (dx, dy) and (-dx, dy); S.triple(dy, right, left, centre) to
    (2, dy), (-2, dy) and (0, dy))."""
    body, inside, pending = [], False, ""
    for line in open(STENCILS):
        if line.startswith("__device__ __forceinline__ void af_sac_%s_adj(" % fam_name):
            inside = True
            continue
        if inside:
            if line.startswith("}"):
                break
            st = (pending + " " + line.strip()).strip() if pending else line.strip()
            if st.startswith(("S.pair(", "S.triple(")) and not st.endswith(";"):
                pending = st  # a statement continued on the next line
                continue
            pending = ""
            body.append(st)

    def run(lGp, lGuv):
        env = {"lGp": lGp, "lGuv": lGuv, "fma": lambda a, b, c: a * b + c, "T": float}
        out, kk = {}, [0.0, 0.0, 0.0]
        names = {"lpK": 0, "luK": 1, "lvK": 2}
        for st in body:
            m = re.match(r"const T (\w+) = (.*);$", st)
            if m:
                env[m.group(1)] = eval(m.group(2), env)
                continue
            m = re.match(r"T (c0\w+)\[3\];", st)
            if m:
                env[m.group(1)] = [0.0, 0.0, 0.0]
                continue
            m = re.match(r"(c0\w+)\[(\d)\] = (.*);$", st)
            if m:
                env[m.group(1)][int(m.group(2))] = eval(m.group(3), env)
                continue
            m = re.match(r"S\.triple\((-?\d+), (.*)\);$", st)
            if m:
                vals = eval("(" + m.group(2) + ")", env)
                dy = int(m.group(1))
                assert len(vals) == 9, st
                for off, part in (((2, dy), vals[:3]), ((-2, dy), vals[3:6]), ((0, dy), vals[6:])):
                    acc = out.setdefault(off, [0.0, 0.0, 0.0])
                    for k in range(3):
                        acc[k] += part[k]
                continue
            m = re.match(r"(lpK|luK|lvK) -= (.*);$", st)
            if m:
                kk[names[m.group(1)]] -= eval(m.group(2), env)
                continue
            m = re.match(r"S\((-?\d+), (-?\d+), (.*)\);$", st)
            if m:
                vals = eval("(" + m.group(3) + ")", env)
                acc = out.setdefault((int(m.group(1)), int(m.group(2))), [0.0, 0.0, 0.0])
                for k in range(3):
                    acc[k] += vals[k]
                continue
            m = re.match(r"S\.pair\((\d+), (-?\d+), (.*)\);$", st)
            if m:
                vals = eval("(" + m.group(3) + ")", env)
                dx, dy = int(m.group(1)), int(m.group(2))
                assert dx > 0 and len(vals) == 6, st
                for off, part in (((dx, dy), vals[:3]), ((-dx, dy), vals[3:])):
                    acc = out.setdefault(off, [0.0, 0.0, 0.0])
                    for k in range(3):
                        acc[k] += part[k]
                continue
            assert st in ("", "}") or st.startswith("{") or st.startswith("//"), st
        return out, kk
    return run


@pytest.mark.parametrize("fam_name", ["V", "EV", "EH", "C"])
def test_generated_transposed_stencils_are_the_adjoint_of_the_tables(fam_name):
    """<lG, G(data)> = <G^T lG, data> for random data and adjoints: the scatter
    code of the adjoint is the exact transpose of the generated forward tables
    (which the previous test pins to the oracle's acoustic operator)."""
    tables = parse_stencils()[fam_name]
    adj = parse_adjoint(fam_name)
    rng = np.random.default_rng(5)
    for trial in range(3):
        lat = {(dx, dy): rng.normal(size=3) for dx in range(-4, 5) for dy in range(-4, 5)}
        K = lat[(0, 0)]
        Gp, Guv = apply_tables(tables, lat, K)
        lGp, lGuv = rng.normal(size=(3, 4)), rng.normal(size=(3, 4))
        lhs = np.sum(lGp * Gp[:, 1:]) + np.sum(lGuv * Guv[:, 1:])
        out, kk = adj(lGp, lGuv)
        rhs = float(np.dot(kk, K))
        for off, vals in out.items():
            rhs += float(np.dot(vals, lat[off]))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)), (trial, lhs, rhs)
