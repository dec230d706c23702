"""Host-side logic of bench.py (no GPU): the staleness guard of the recorded ncu
traffic (a hash of the fused kernel's code, blind to comments), the scaling of
that traffic to a launch, and the per-field relative L-inf of FP32 against FP64
(velocity and momentum taken as vectors); the clock summary of the sampled
nvidia-smi lines; the marshalling of state arrays into the ABI's 16 planes."""
import os
import shutil

import numpy as np
import pytest

import bench


def _copy_sources(tmp_path):
    for f in bench.FUSED_SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)
    return tmp_path


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    root = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.fused_source_hash()
    target = root / bench.FUSED_SOURCES[0]
    text = target.read_text()
    target.write_text("// a new leading comment\n/* and a block\n   comment */\n\n" +
                      text.replace("\n", "\n   ", 1))
    assert bench.fused_source_hash() == h0
    target.write_text(text.replace("constexpr int FUSED_TX", "constexpr int  FUSED_TX", 1)
                      .replace("FUSED_TY = AF_FUSED_TY", "FUSED_TY = AF_FUSED_TY + 0", 1))
    assert bench.fused_source_hash() != h0


def _recorded_hash():
    with open(os.path.join(bench.ROOT, bench.PROFILE)) as f:
        for line in f:
            if line.startswith("kernel_source_sha256_16:"):
                return line.split(":", 1)[1].strip()
    return None


def test_recorded_traffic_scales_to_a_launch(monkeypatch):
    # as if the kernel sources were those the committed profile was captured from
    monkeypatch.setattr(bench, "fused_source_hash", _recorded_hash)
    full = bench.profiled_traffic(4194304)
    assert full is not None and full > 0
    assert abs(bench.profiled_traffic(2 * 4194304) - 2 * full) < 1e-6 * full


def test_recorded_traffic_is_dropped_when_the_kernel_changed(monkeypatch):
    monkeypatch.setattr(bench, "fused_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic(4194304) is None


def test_per_field_error_takes_velocity_as_a_vector():
    rng = np.random.default_rng(0)
    b = 1.0 + rng.random((16, 6, 5))
    b[[1, 5, 9, 13]] = 1.0   # u (and rho u) = 1
    b[[2, 6, 10, 14]] = 0.0  # v (and rho v) = 0: a per-plane form would divide by 0
    a = b.copy()
    a[6] += 1e-3              # v error at the vertices
    a[3] *= 1 + 2e-4          # energy average
    # velocity error 1e-3 against |velocity| 1; energy 2e-4 of itself
    assert abs(bench.rel_linf_fields(a, b) - 1e-3) < 1e-12
    a[6] = b[6]
    assert abs(bench.rel_linf_fields(a, b) - 2e-4) < 1e-12


def test_clock_summary_from_sampled_lines():
    s = bench.ClockSampler(0)
    s.lines = ["2070, 2070, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, Not Active, Not Active, Not Active, Active",
               "2070, 2070, Not Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3, "source": None}
    s.lines = ["1500, 2070, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None,
                                               "reasons": [], "samples": 0, "source": None}


def test_state_planes_are_marshalled_in_the_documented_order():
    import paper_2605_12915_gb300 as af
    arr = np.zeros((16, 3, 5))
    ptr, dev = af._array_ptr(arr)
    assert ptr == arr.ctypes.data and not dev
    st = af._state_struct(ptr, 15)
    planes = list(st.avg) + list(st.vtx) + list(st.ev) + list(st.eh)
    assert planes == [ptr + 8 * 15 * p for p in range(16)]
    with pytest.raises(AssertionError):
        af._array_ptr(np.zeros((16, 3, 5), dtype=np.float32))
    with pytest.raises(AssertionError):
        af._array_ptr(np.zeros((16, 5, 3)).transpose(0, 2, 1))
