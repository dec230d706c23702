"""Benchmark: cell-updates/s of the RB-TAI Active Flux step on the 2048^2
low-Mach doubly periodic shear layer (FP32 bulk arithmetic, compensated
averages, FP64 invariants), one JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value      device-timed cell-updates/s of K steps (CUDA events on the solver's
           stream), state resident in HBM; summed over ranks for N > 1
           (independent replicas, max-over-ranks time).
e2e        the same metric through the public API with host buffers: every step
           copies its state in from pinned host memory, advances it and copies
           the result back out (af_exchange_state overlaps one step's outgoing
           copy with the next step's incoming one; af_exchange_state_async
           enqueues it all, so that consecutive steps' transfers queue back to
           back); the run ends with a get of the last result, which waits for
           every transfer; the median of three timed runs (max over ranks).
           sync_exchange_ms_per_step: the same with af_exchange_state, which
           returns with the new state in place.  link_ms_per_step: the same
           transfers alone (both directions at once, no compute), the bound of
           this leg.
roofline   the dominant kernel (the fused step kernel), timed per launch with CUDA
           events: its algorithmic FP32 lane operations per launch / duration
           against 152 SMs x 128 FP32 lanes x SM clock ("alu", the bound), and
           inside it ("hbm") the algorithmic bytes per launch / duration against
           the measured HBM peak.
fp64       FP64 throughput of the same workload, its fraction of a measured FP64
           rate, and FP32 against FP64 after 100 steps (per field and per plane).
fp32_plain the same workload with plain FP32 averages (no lo words).
shear2000  the workload at its stated length, 2000 steps: throughput, drift of
           the conserved totals, change of the entropy functional.
ensemble   the 256-grid vortex ensemble, one batched launch per step against
           per-grid launches.
adjoint    the discrete adjoint step against the forward step.
foot_centred  context: the FP64 step with the foot-centred point update
           against the FP64 transported step on a 128^2 copy.
cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload.
--impl reference  times the oracle itself (this workload has no other
           reference implementation), on rank 0 only.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s on 2048^2 Euler AF, FP32 vs FP64 at stated L-inf; % HBM peak"
UNIT = "cell-updates/s"
N_CELLS_SIDE = 2048


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32_comp", choices=["fp32", "fp32_comp", "fp64"])
    p.add_argument("--n", type=int, default=N_CELLS_SIDE)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=50)
    p.add_argument("--kernel-reps", type=int, default=20)
    p.add_argument("--fp64-steps", type=int, default=100,
                   help="steps of the FP64 comparison run (0: skip)")
    p.add_argument("--no-ensemble", action="store_true",
                   help="skip the batched 256-grid vortex ensemble (200 steps)")
    p.add_argument("--shear-steps", type=int, default=2000,
                   help="steps of the full-length shear-layer run (conservation drift and "
                        "entropy; 0: skip)")
    p.add_argument("--no-fc", action="store_true",
                   help="skip the cost of the foot-centred variant (context)")
    p.add_argument("--fp32-steps", type=int, default=200,
                   help="steps of the plain FP32 (uncompensated) leg (0: skip)")
    p.add_argument("--adjoint-steps", type=int, default=5,
                   help="adjoint steps timed against the forward step (0: skip)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP32 arithmetic operations of one cell-update of the fused step, counted
# from the code (add, subtract, multiply, fused multiply-add, reciprocal,
# reciprocal square root and floor count once each; comparisons, clamps,
# conversions and index arithmetic do not count; no halo recomputation):
# centre recovery 184, freezing of the 4 nodes 36, acoustic stencils 695
# (generated), increment mixing and the two Horner evaluations of 4 nodes 160,
# six point updates of 144, space-time Simpson fluxes of 2 edges 278,
# compensated average update 148.
ALU_OPS_PER_CELL = 2365
# plain FP32 averages: the compensated update (148) is replaced by four
# three-term updates of the averages (16)
ALU_OPS_PER_CELL_PLAIN = 2365 - 148 + 16
FUSED_SOURCES = ["paper_2605_12915_gb300/csrc/af_fused.cuh",
                 "paper_2605_12915_gb300/csrc/af_common.cuh",
                 "paper_2605_12915_gb300/csrc/af_stencils.cuh",
                 "paper_2605_12915_gb300/csrc/af_ref_kernels.cuh"]
PROFILE = "profiles/k_fused_step_pipe_shear2048_fp32comp.md"


def fused_kernel_name(nx, ny):
    """The FP32 step kernel the library launches for an nx x ny grid: the
    persistent pipelined kernel when the grid allows it and AF_PIPE is not 0."""
    if os.environ.get("AF_PIPE") == "0" or nx % 4 or nx < 40 or ny < 38:
        return "k_fused_step"
    return "k_fused_step_pipe"


def fused_source_hash():
    """Hash of the fused kernel's code (comments, blank lines and indentation
    removed, so that documentation edits keep a recorded profile valid)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for line in text.splitlines():
            line = line.split("//", 1)[0].strip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(n_cells):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    scaled to n_cells; None if the kernel source changed since the capture."""
    try:
        kv = {}
        with open(os.path.join(ROOT, PROFILE)) as f:
            for line in f:
                if ":" in line and not line.startswith(("|", "#", " ")):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != fused_source_hash():
            return None
        return float(kv["traffic_bytes_per_launch"]) * n_cells / float(kv["cells_per_launch"])
    except Exception:
        return None


# NVML clock-event reason bits (nvml.h, nvmlClocksEventReason*)
_NVML_REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
                 "sw_power_cap": 0x4}


class ClockSampler:
    """SM clocks and throttle reasons sampled during a timed region: NVML read
    directly (ctypes, every `period_s`) when the driver's library is there, else
    `nvidia-smi -lms 100`.  Both record lines "sm, max, hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap" ("Active" /
    "Not Active"), summarised by summary()."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, uuid=None, period_s=0.002):
        self.index = index
        self.uuid = uuid
        self.period_s = period_s
        self.proc = None
        self.thread = None
        self.stop = None
        self.source = None
        self.lines = []

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        ok = False
        if self.uuid:
            ok = lib.nvmlDeviceGetHandleByUUID(("GPU-" + str(self.uuid)).encode(),
                                               ctypes.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        return lib, h

    def _poll_nvml(self, lib, h):
        import ctypes
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    get_reasons(h, ctypes.byref(rs)) == 0):
                flags = ["Active" if rs.value & _NVML_REASONS[k] else "Not Active"
                         for k in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                   "sw_power_cap")]
                self.lines.append(", ".join([str(clk.value), str(mx.value)] + flags))
            self.stop.wait(self.period_s)

    def __enter__(self):
        import threading as th
        try:
            lib, h = self._nvml_handle()
            self.stop = th.Event()
            self.thread = th.Thread(target=self._poll_nvml, args=(lib, h), daemon=True)
            self.thread.start()
            self.source = "nvml"
            return self
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            self.source = "nvidia-smi"
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.stop is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sm),
                "source": self.source}


def aggregate(ms_local, n_cells, steps, world, device):
    """Whole-job throughput of N independent replicas: the slowest rank's time
    (max over ranks) and the cells all ranks advanced per second."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, n_cells * steps * world / (ms * 1e-3)


def dist_setup(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def _oracle_replica(sample_n, sample_steps, barrier, results):
    """One copy of the oracle sample in its own process (all cores leg)."""
    import oracle
    from workloads import inputs as I
    S = I.shear(n=sample_n)
    barrier.wait()
    t = time.perf_counter()
    oracle.run(S.state, S.grid.h, S.gamma, S.dt, sample_steps)
    results.put(time.perf_counter() - t)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(P, sample_n=512, sample_steps=6, all_cores=True):
    """The oracle as it stands on a bounded sample of the same workload: the same
    shear layer on a sample_n^2 grid, sample_steps steps, one host core; and, as
    `all_cores`, one such copy per host core run at the same time (independent
    processes, started by spawn: the oracle is single-threaded and unmodified),
    their cell-updates summed over the slowest copy's time."""
    import oracle
    from workloads import inputs as I
    S = I.shear(n=sample_n)
    t = time.perf_counter()
    oracle.run(S.state, S.grid.h, S.gamma, S.dt, sample_steps)
    el = time.perf_counter() - t
    out = {"value": sample_n * sample_n * sample_steps / el, "unit": UNIT, "cores": 1,
           "kind": "oracle",
           "sample": "shear layer %d^2, %d steps, FP64 oracle, 1 thread (%.1f s)"
                     % (sample_n, sample_steps, el)}
    if all_cores:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        n = host_cores()
        barrier, results = ctx.Barrier(n), ctx.Queue()
        procs = [ctx.Process(target=_oracle_replica, args=(sample_n, sample_steps, barrier, results))
                 for _ in range(n)]
        for p in procs:
            p.start()
        times = [results.get() for _ in range(n)]
        for p in procs:
            p.join()
        slow = max(times)
        out["all_cores"] = {"value": n * sample_n * sample_n * sample_steps / slow, "unit": UNIT,
                            "cores": n, "kind": "oracle",
                            "sample": "%d copies of the sample at once, one process per core "
                                      "(slowest %.1f s)" % (n, slow)}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from workloads import inputs as I
    oracle.build()
    n = 128  # bounded sample per step: a 128^2 copy of the workload
    S = I.shear(n=n)
    st = S.state
    for _ in range(args.warmup):
        st, _ = oracle.step(st, S.grid.h, S.gamma, S.dt)
    t = time.perf_counter()
    for _ in range(args.steps):
        st, _ = oracle.step(st, S.grid.h, S.gamma, S.dt)
    el = time.perf_counter() - t
    v = n * n * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "low-Mach shear layer (FP64 CPU oracle, %d^2 sample per step)" % n,
                       "n": n, "cfl": 0.4},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "shear layer %d^2 per step, %d steps" % (n, args.steps)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2605_12915_gb300 as af
    from workloads import inputs as I

    rank, world, local = dist_setup(args)
    af._build.build()
    af.load()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    n_sms = props.multi_processor_count
    uuid = getattr(props, "uuid", None)
    P = I.shear(n=args.n)
    N = P.grid.nx * P.grid.ny
    stream = torch.cuda.Stream()
    dev_state = torch.from_numpy(P.state).cuda()
    torch.cuda.synchronize()
    solver = af.Solver(P.grid, P.gamma, dev_state, precision=args.precision, stream=stream)
    inv0 = solver.invariants()

    # warm-up
    solver.step(P.dt, args.warmup)
    solver.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, uuid) as clocks:
        ev0.record(stream)
        solver.step(P.dt, args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    solver.sync()
    ms, value = aggregate(ms, N, args.steps, world, "cuda")
    inv1 = solver.invariants()

    # dominant kernel: per-launch duration of the step kernel(s)
    fused = args.precision != "fp64" and os.environ.get("AF_PATH", "fused") != "ref"
    kstats = solver_kernel_stats(af, solver, P, stream, torch, max(1, args.kernel_reps), fused)

    # end to end through the public API with pinned host buffers
    host_in = torch.from_numpy(P.state.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_steps = max(1, args.e2e_steps)

    def e2e_run(n, exchange):
        # every step's input goes in and its result comes out; one call hands a
        # step's result out while the next step's input comes in, the two
        # transfers overlapping on the link (and the result's with the next step);
        # the final get waits for every transfer of the run
        solver.set_state(host_in)
        for i in range(n):
            solver.step(P.dt, 1)
            if i + 1 < n:
                exchange(host_out, host_in)
            else:
                solver.state(host_out)
        torch.cuda.synchronize()

    def e2e_runs(exchange):
        e2e_run(2, exchange)  # first use allocates the staging buffers and streams
        # three timed runs, the median (the host side of the link is shared with
        # other work on the node and varies from run to run)
        runs = []
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            e2e_run(e2e_steps, exchange)
            runs.append(time.perf_counter() - t0)
        return runs

    # af_exchange_state_async (the exchange enqueued, so that consecutive steps'
    # transfers queue back to back) and, beside it, af_exchange_state (returns
    # with the new state in place)
    runs = e2e_runs(solver.exchange_async)
    runs_sync = e2e_runs(solver.exchange)
    e2e_ms, e2e_value = aggregate(1e3 * sorted(runs)[1], N, e2e_steps, world, "cuda")
    sync_ms, _ = aggregate(1e3 * sorted(runs_sync)[1], N, e2e_steps, world, "cuda")
    link_ms = link_copy_ms(torch, host_in, host_out)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(host_in.numel() * 8),
           "d2h_bytes_per_step": int(host_out.numel() * 8),
           "ms_per_step": e2e_ms / e2e_steps, "steps": e2e_steps,
           "runs_ms_per_step": [round(1e3 * r / e2e_steps, 3) for r in runs],
           "api": "af_exchange_state_async per step (host planes, pinned); the run "
                  "ends with af_get_state, which waits for every transfer",
           "sync_exchange_ms_per_step": sync_ms / e2e_steps,
           "link_ms_per_step": link_ms,
           "link_frac": link_ms / (e2e_ms / e2e_steps),
           "link_note": "link_ms_per_step: one step's input planes copied in and its result "
                        "copied out at the same time (plain copies of the same pinned buffers, "
                        "no compute); link_frac = that time / the e2e step time"}

    hbm, peak_kind = peaks()
    bytes_per_cell = {"fp32": 128, "fp32_comp": 160, "fp64": 256}[args.precision]
    ach = bytes_per_cell * N / (kstats["ms_per_launch"] * 1e-3) / 1e9
    csum = clocks.summary()
    sm_hz = 1e6 * (csum["sm_max_mhz"] or 2070.0)
    alu_peak = n_sms * 128 * sm_hz / 1e12
    alu_ach = ALU_OPS_PER_CELL * N / (kstats["ms_per_launch"] * 1e-3) / 1e12
    hbm_part = {"achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_kind": peak_kind, "bytes_per_cell": bytes_per_cell}
    if fused:
        # FP32 stencil arithmetic on the CUDA cores binds the fused kernel (DRAM
        # runs near a tenth of its peak)
        roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "T FP32 op/s",
                "frac": alu_ach / alu_peak, "ops_per_cell": ALU_OPS_PER_CELL,
                "peak_kind": "%d SMs x 128 FP32 lanes x max SM clock" % n_sms,
                "traffic": profiled_traffic(N), "kernel": kstats["kernel"], "hbm": hbm_part}
    else:
        roof = dict(bound="hbm", traffic=None, kernel=kstats["kernel"], **hbm_part)
    extras = world == 1  # replicas (N > 1) time the step only
    fp64 = fp64_compare(af, I, P, solver_state_after(af, P, args, stream), args, stream, torch) \
        if args.fp64_steps > 0 and extras else None
    adjoint = adjoint_cost(af, P, args, stream, torch, kstats["ms_per_launch"]) \
        if args.adjoint_steps > 0 and extras else None
    ensemble = ensemble_block(af, I, stream, torch) if not args.no_ensemble and extras else None
    shear_long = shear_long_run(af, P, args.shear_steps, stream, torch, local, uuid) \
        if args.shear_steps > 0 and extras else None
    fp32_plain = plain_fp32_leg(af, P, args.fp32_steps, stream, torch, alu_peak, hbm) \
        if args.fp32_steps > 0 and extras and args.precision == "fp32_comp" else None
    foot_centred = foot_centred_cost(af, I, stream, torch) if extras and not args.no_fc else None
    drift = (inv1[:4] - inv0[:4]) / np.array([inv0[0], inv0[0], inv0[0], inv0[3]])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp32_comp": "f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "low-Mach doubly periodic shear layer, %d^2 cells, CFL 0.4, "
                                   "RB-TAI, %s" % (args.n, args.precision),
                       "n": args.n, "precision": args.precision, "variant": "tai",
                       "l2": "inputs larger than L2 (state %.0f MB)" % (bytes_per_cell * N / 2 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roof,
            "e2e": e2e,
            # the steps' kernels, and the one that copies the error word to the
            # host at the end of the af_step call
            "gpu_launches": kstats["launches_per_step"] * args.steps + 1,
            "clocks": csum,
            "fp64": fp64,
            "adjoint": adjoint,
            "ensemble": ensemble,
            "fp32_plain": fp32_plain,
            "foot_centred": foot_centred,
            "shear2000": shear_long,
            "conservation_drift": [float(x) for x in drift],
            "entropy_change": float(inv1[4] - inv0[4])}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(P)
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ensemble_block(af, I, stream, torch, n_problems=256, steps=200):
    """Seeded ensemble of isentropic vortices on grids of 64^2..512^2 cells, FP32:
    one batched, graph-captured launch per step against per-grid launches."""
    specs = I.ensemble(n_problems, seed=0, n_steps=steps)
    probs = [I.ensemble_member(sp) for sp in specs]
    dts = [p.dt for p in probs]
    cells = sum(p.grid.nx * p.grid.ny for p in probs)
    b = af.Batch(probs, precision="fp32", stream=stream)
    b.step(dts, 1)  # tunes the tile geometry
    b.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(dts, steps)
    e1.record(stream)
    e1.synchronize()
    b.sync()
    ms_batch = e0.elapsed_time(e1)
    geom, tune = b.info()
    b.close()
    solvers = [af.Solver(p.grid, p.gamma, p.state, precision="fp32", stream=stream) for p in probs]
    for s, dt in zip(solvers, dts):
        s.step(dt, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for s, dt in zip(solvers, dts):
        s.step(dt, steps)
    e1.record(stream)
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for s in solvers:
        s.sync()
        s.close()
    return {"problems": n_problems, "cells": cells, "steps": steps,
            "batched": {"value": cells * steps / (ms_batch * 1e-3), "unit": UNIT, "ms": ms_batch,
                        "tile_geometry": ["32x32/512 per tile", "24x16/256x2 per tile",
                                          "16x16/256x3 per tile",
                                          "32x32/512 persistent, staged"][geom],
                        "tune_ms_per_step": tune},
            "sequential": {"value": cells * steps / (ms_seq * 1e-3), "unit": UNIT, "ms": ms_seq},
            "speedup": ms_seq / ms_batch}


def shear_long_run(af, P, steps, stream, torch, local, uuid):
    """The shear-layer workload at its stated length (2000 steps from the initial
    state, FP32 with compensated averages): device-timed throughput, the drift
    of the conserved totals and the change of the entropy functional (FP64
    reductions of the initial and final states)."""
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32_comp", stream=stream)
    inv0 = s.invariants()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, uuid, period_s=0.01) as clk:
        e0.record(stream)
        s.step(P.dt, steps)
        e1.record(stream)
        e1.synchronize()
    s.sync()
    ms = e0.elapsed_time(e1)
    inv1 = s.invariants()
    s.close()
    N = P.grid.nx * P.grid.ny
    names = af.INVARIANT_NAMES
    # drift relative to the initial totals; the momentum totals are zero, so
    # their drift is stated relative to the total mass
    scale = [inv0[0], inv0[0], inv0[0], inv0[3]]
    return {"steps": steps, "t_final": steps * P.dt, "ms_per_step": ms / steps,
            "value": N * steps / (ms * 1e-3), "unit": UNIT, "precision": "fp32_comp",
            "conservation_drift": {names[k]: float((inv1[k] - inv0[k]) / scale[k])
                                   for k in range(4)},
            "entropy": {k: {"initial": float(inv0[i]), "final": float(inv1[i]),
                            "change": float(inv1[i] - inv0[i])}
                        for k, i in (("simpson", 4), ("average", 5))},
            "kinetic_energy": {"initial": float(inv0[6]), "final": float(inv1[6])},
            "min_rho": float(inv1[8]), "min_p": float(inv1[9]),
            "clocks": clk.summary()}


def foot_centred_cost(af, I, stream, torch, n=128, steps=3):
    """Context, not a target: the FP64 step with the foot-centred point update
    (Appendix C) against the FP64 transported step, same shear layer at n^2."""
    P = I.shear(n=n)
    out = {"n": n, "steps": steps}
    for variant in ("fc", "tai"):
        s = af.Solver(P.grid, P.gamma, P.state, precision="fp64", variant=variant, stream=stream)
        s.step(P.dt, 1)
        s.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(P.dt, steps)
        e1.record(stream)
        e1.synchronize()
        s.sync()
        s.close()
        out[variant + "_fp64_ms_per_step"] = e0.elapsed_time(e1) / steps
    out["cost_ratio"] = out["fc_fp64_ms_per_step"] / out["tai_fp64_ms_per_step"]
    return out


def plain_fp32_leg(af, P, steps, stream, torch, alu_peak, hbm):
    """The same workload with plain FP32 averages (no lo words): per-launch time
    of the fused kernel and its fractions of the FP32-issue and HBM rooflines
    (128 algorithmic bytes per cell)."""
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp32", stream=stream)
    s.step(P.dt, 5)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(P.dt, steps)
    e1.record(stream)
    e1.synchronize()
    s.sync()
    s.close()
    ms = e0.elapsed_time(e1) / steps
    N = P.grid.nx * P.grid.ny
    alu = ALU_OPS_PER_CELL_PLAIN * N / (ms * 1e-3) / 1e12
    gbs = 128 * N / (ms * 1e-3) / 1e9
    return {"ms_per_step": ms, "value": N / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "alu": {"achieved": alu, "peak": alu_peak, "frac": alu / alu_peak,
                    "ops_per_cell": ALU_OPS_PER_CELL_PLAIN, "unit": "T FP32 op/s"},
            "hbm": {"achieved": gbs, "peak": hbm, "frac": gbs / hbm, "bytes_per_cell": 128,
                    "unit": "GB/s"}}


def link_copy_ms(torch, host_in, host_out, reps=3):
    """Time of one step's host transfers alone: the input planes copied from
    pinned host memory to the device while the previous result is copied back
    (two streams, both directions at once), best of `reps`."""
    d_in = torch.empty(host_in.shape, dtype=host_in.dtype, device="cuda")
    d_out = torch.empty(host_out.shape, dtype=host_out.dtype, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    best = float("inf")
    for _ in range(reps + 1):  # the first pass warms up the streams
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s_in):
            d_in.copy_(host_in, non_blocking=True)
        with torch.cuda.stream(s_out):
            host_out.copy_(d_out, non_blocking=True)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    del d_in, d_out
    return 1e3 * best


def adjoint_cost(af, P, args, stream, torch, fwd_ms):
    """Time of one discrete adjoint step (af_adjoint_step, device buffers, same
    precision and workload) against one forward step."""
    s = af.Solver(P.grid, P.gamma, P.state, precision=args.precision, stream=stream)
    # a seeded normal adjoint state (lambda = 1 everywhere costs the same: the
    # kernels skip no work on it, measured 3.529 against 3.530 ms at 2048^2)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    lam = torch.randn((16, P.grid.ny, P.grid.nx), dtype=torch.float64, device="cuda",
                      generator=gen)
    out = torch.empty_like(lam)
    s.adjoint(P.dt, lam, out)  # allocates the adjoint work planes
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.adjoint_steps):
        s.adjoint(P.dt, lam, out)
    e1.record(stream)
    e1.synchronize()
    s.close()
    ms = e0.elapsed_time(e1) / args.adjoint_steps
    return {"ms_per_step": ms, "forward_ms_per_step": fwd_ms, "ratio": ms / fwd_ms,
            "note": "adjoint step = recomputation of the step's intermediates (fused kernel in "
                    "the FP32 modes) + reverse sweep, including the FP64 conversion of the "
                    "adjoint state in and out"}


def solver_state_after(af, P, args, stream):
    """FP32 state after args.fp64_steps steps from the initial state."""
    s = af.Solver(P.grid, P.gamma, P.state, precision=args.precision, stream=stream)
    s.step(P.dt, args.fp64_steps)
    out = s.state()
    s.close()
    return out


def fp64_compare(af, I, P, st32, args, stream, torch):
    """FP64 throughput of the same workload (unfused FP64 kernels) and the
    FP32-vs-FP64 relative L-inf per plane (max |a-b| / max |b|) after the same
    number of steps."""
    s = af.Solver(P.grid, P.gamma, P.state, precision="fp64", stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(P.dt, args.fp64_steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.fp64_steps
    st64 = s.state()
    e0.record(stream)
    s.invariants()
    e1.record(stream)
    e1.synchronize()
    inv_ms = e0.elapsed_time(e1)
    s.close()
    num = np.max(np.abs(st32 - st64), axis=(1, 2))
    den = np.maximum(np.max(np.abs(st64), axis=(1, 2)), 1e-300)
    N = P.grid.nx * P.grid.ny
    peak = fp64_peak(torch)
    ach = ALU_OPS_PER_CELL_PLAIN * N / (ms * 1e-3) / 1e12
    return {"value": N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": args.fp64_steps,
            "roofline": {"bound": "fp64 alu", "achieved": ach, "unit": "T FP64 op/s",
                         "ops_per_cell": ALU_OPS_PER_CELL_PLAIN, "peak": peak,
                         "frac": ach / peak if peak else None,
                         "peak_kind": "measured: torch float64 matmul 4096^3 (cuBLAS), "
                                      "multiply-adds counted once"},
            "invariants_ms": inv_ms,
            "fp32_vs_fp64_rel_linf": rel_linf_fields(st32, st64),
            "fp32_vs_fp64_rel_linf_per_plane_max": float(np.max(num / den)),
            "fp32_vs_fp64_rel_linf_per_plane": [float(x) for x in num / den]}


def fp64_peak(torch, n=4096, reps=3):
    """Measured FP64 rate of this GPU in T multiply-adds/s (a multiply-add
    counted once, like the operation counts): the best of `reps` float64
    matmuls of n^3 through cuBLAS."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return float(n) ** 3 / (best * 1e-3) / 1e12


def rel_linf_fields(a, b):
    """Relative L-inf per field, max over fields: density, pressure, energy and
    mass averages each on their own; velocity (u, v) and momentum (rho u, rho v)
    as vectors, normalised by their largest magnitude."""
    def rel(ix, vec=False):
        d = np.abs(a[ix] - b[ix])
        if vec:
            return float(np.max(np.sqrt(np.sum(d * d, axis=0))) /
                         max(np.max(np.sqrt(np.sum(b[ix] ** 2, axis=0))), 1e-300))
        return float(np.max(d) / max(np.max(np.abs(b[ix])), 1e-300))
    errs = [rel([0]), rel([1, 2], True), rel([3])]
    for base in (4, 8, 12):
        errs += [rel([base]), rel([base + 1, base + 2], True), rel([base + 3])]
    return max(errs)


def solver_kernel_stats(af, solver, P, stream, torch, reps, fused):
    """Mean duration of one step's launches (the single fused kernel when that
    path is active), timed with CUDA events on the solver's stream."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for r in range(reps):
        solver.step(P.dt, 1)
        ev[r + 1].record(stream)
    ev[-1].synchronize()
    ts = [ev[r].elapsed_time(ev[r + 1]) for r in range(reps)]
    if fused:
        return {"ms_per_launch": float(np.mean(ts)),
                "kernel": fused_kernel_name(P.grid.nx, P.grid.ny), "launches_per_step": 1}
    return {"ms_per_launch": float(np.mean(ts)), "kernel": "all 10 launches of one step",
            "launches_per_step": 10}


if __name__ == "__main__":
    main()
