"""Benchmark of the LBRS time step on one GB300 (or one grid split over N GPUs under torchrun).

Workload: the 2-D D2Q4 four-quadrant Riemann problem, 1024 x 1024 cells on
[0, 1]^2, quadrant states from seed 0 (rho ~ U[0.1, 1.5], p ~ U[0.03, 1.5],
u, v ~ U[-1.2, 1.2]), transmissive boundaries, gamma = 1.4, omega = 1,
FP32 distributions.  One bench "step" is one LBRS time step over the whole
grid (stream, boundary conditions, moments, fluxes, equilibria, relaxation).

Printed: one JSON line with MLUPS (million lattice updates per second) of the
FP32 path, timed as calls of three time steps (one launch of the three-steps-
per-launch kernel) with the L2 cache flushed before every call, the FP64 path's
MLUPS and the FP32 density L1 error after the configuration's 1000 steps,
the HBM roofline of the step kernel, an end-to-end figure through the public
API with host buffers, and the FP64 CPU oracle timed on the host cores.

Under torchrun with N > 1 ranks the same grid is split into N y-slabs, one per GPU, whose
cut rows are exchanged with NCCL send/recv every three steps (strong scaling; see run_slabs).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "2D LBRS MLUPS FP32 vs FP64 at stated L1 error; % HBM roofline; adjoint/fwd cost"
UNIT = "MLUPS"
BYTES_PER_LUP_F32 = 128      # 16 FP32 distributions read + 16 written per cell and step
BYTES_PER_LUP_F32_FUSED2 = 64  # two steps per launch: the 128 B per cell are read and written once per two steps
BYTES_PER_LUP_F32_FUSED3 = 128 / 3   # three steps per launch: once per three steps
SLAB_HALO = 3                 # ghost rows per cut with N > 1 GPUs: one exchange per three-step launch
BYTES_PER_LUP_F64 = 256
BYTES_PER_LUP_F16NEQ = 80     # U (4 x FP32) + 12 FP16 non-equilibrium parts, read + written
BYTES_PER_LUP_F32U = 32       # omega = 1 moments-only form: U (4 x FP32), read + written
L2_FLUSH_BYTES = 256 << 20   # twice the 129 MB L2
CONFIG_STEPS = 1000


def workload():
    """The headline configuration (workloads/configs/quadrant_riemann_1024.json)."""
    return workloads.from_config("quadrant_riemann_1024")[1]


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def config_dict(wl, extra=None):
    d = {"workload": "2-D D2Q4 four-quadrant Riemann 1024x1024, seed 0, transmissive, 1000-step configuration",
         "config_file": "workloads/configs/quadrant_riemann_1024.json",
         "nx": wl.nx, "ny": wl.ny, "lattice": "D2Q4", "gamma": wl.gamma, "omega": wl.omega,
         "lambda": wl.lam,
         "l2": "flushed (256 MiB write) before every timed call of lbrs_step (three time steps for the "
               "FP32 headline, one for the others), outside the call's CUDA events"}
    if extra:
        d.update(extra)
    return d


def parallelism(ws: int) -> str:
    return "1 GPU" if ws == 1 else (f"{ws} y-slabs, one per GPU, {SLAB_HALO} ghost rows per cut, NCCL send/recv "
                                    f"of the rows every {SLAB_HALO} steps")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_source_sha() -> str:
    """Hash of the code that defines the three-step kernel's launches: the shared device helpers, the FP32
    kernel file up to the end of the three-step kernel (everything it uses is defined above it; the scalar
    lattice's section follows it), and the three-step launcher with its tensor map and prefetch distance.
    Changes elsewhere (the scalar and adjoint kernels, other launchers) leave the traffic record valid."""
    csrc = os.path.join(ROOT, "paper_1504_07034_gb300", "csrc")
    with open(os.path.join(csrc, "lbrs_kernels.cuh"), "rb") as fh:
        cuh = fh.read()
    with open(os.path.join(csrc, "lbrs_kernels_f32.cu"), "rb") as fh:
        f32 = fh.read()
    end = f32.find(b"// ---------------------------------------------------------------- scalar D2Q4, two steps per launch")
    a = f32.find(b"// The distance of the three-step kernel's L2 prefetch")
    b = f32.find(b"cudaError_t launch_step2_f32(")
    parts = (cuh, f32[:end], f32[a:b]) if min(end, a, b) >= 0 and a < b else (cuh, f32)   # markers moved: all
    h = hashlib.sha256()
    for part in parts:
        h.update(part)
    return h.hexdigest()[:16]


def measured_traffic(cells: int):
    """DRAM bytes per launch of the FP32 three-step kernel from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "step2d_f32_fused3_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != kernel_source_sha():
        return None
    return rec["dram_bytes_per_launch"] * cells / rec["cells"]


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 20 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        self.t0 = time.time()
        return self

    def stop(self):
        if not self.proc:
            return []
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        return rows

    def __exit__(self, *a):
        return False


def summarise_clocks(rows):
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(wl, seconds=12.0):
    """The FP64 oracle as it stands on the host cores: MLUPS over a bounded number of steps."""
    import oracle
    o = oracle.Oracle.from_workload(wl)
    fs = o.init(o.prim_to_cons(wl.prim))
    fs, t1 = o.timed_run(fs, 2)
    n = max(2, min(wl.steps, int(seconds / max(t1 / 2, 1e-6))))
    _, t = o.timed_run(fs, n)
    out = {"value": wl.cells * n / t / 1e6, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
           "sample": f"FP64 C oracle, full {wl.nx}x{wl.ny} grid, steps 3..{n + 2} of the 1000-step run "
                     f"({t:.1f} s, OpenMP over rows)"}
    # the same oracle on one thread, a few steps of the same run
    o1 = oracle.Oracle.from_workload(wl, nthreads=1)
    _, t1 = o1.timed_run(fs, 1)
    n1 = max(1, min(wl.steps, int(0.4 * seconds / max(t1, 1e-6))))
    _, t1 = o1.timed_run(fs, n1)
    out["single_thread"] = {"value": wl.cells * n1 / t1 / 1e6, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} steps of the same grid ({t1:.1f} s)"}
    return out


def _oracle_rate(o, fs, cells, seconds, max_steps):
    """MLUPS of the oracle `o` from fs over about `seconds` of steps (at most max_steps)."""
    _, t1 = o.timed_run(fs, 1)
    n = max(1, min(max_steps, int(seconds / max(t1, 1e-6))))
    _, t = o.timed_run(fs, n)
    return cells * n / t / 1e6, n, t


def oracle_per_config(seconds=4.0):
    """The FP64 oracle as it stands, on the host cores and on one thread, beside each seeded
    configuration other than the headline: bounded samples of each (a few seconds of CPU
    work apiece), with the full run's time extrapolated from the sample where the sample
    is not the whole run."""
    import oracle
    out = {}
    # 1: Sod, the whole run
    cfg, wl = workloads.from_config("sod_d1q2_1000")
    res = {"workload": cfg["name"], "steps": wl.steps}
    for name, nth in (("all_cores", 0), ("one_thread", 1)):
        o = oracle.Oracle.from_workload(wl, nthreads=nth)
        fs = o.init(o.prim_to_cons(wl.prim))
        _, t = o.timed_run(fs, wl.steps)
        res[name] = {"value": wl.nx * wl.steps / t / 1e6, "unit": UNIT, "seconds": t,
                     "cores": oracle.max_threads() if nth == 0 else 1, "sample": "the whole run"}
    out["sod_d1q2_1000"] = res
    # 3: oblique shock, the first steps of the run, the 20000-step time extrapolated
    cfg, wl = workloads.from_config("oblique_shock_4096x1024", steps=0)
    full_steps = cfg["kwargs"]["steps"]
    res = {"workload": cfg["name"]}
    for name, nth, sec in (("all_cores", 0, 2 * seconds), ("one_thread", 1, seconds)):
        o = oracle.Oracle.from_workload(wl, nthreads=nth)
        fs = o.init(o.prim_to_cons(wl.prim))
        v, n, t = _oracle_rate(o, fs, wl.cells, sec, 2000)
        res[name] = {"value": v, "unit": UNIT, "cores": oracle.max_threads() if nth == 0 else 1,
                     "sample": f"steps 2..{n + 1} of the run on the full grid ({t:.1f} s)",
                     "extrapolated_full_run_s": wl.cells * full_steps / (v * 1e6), "extrapolated": True}
    out["oblique_shock_4096x1024"] = res
    # 4: batched tubes, whole tubes from the front of the batch up to a bounded number of updates
    cfg, tb = workloads.from_config("batched_tubes_4096")
    budget, done, t = 2e8, 0, 0.0
    b = 0
    import time as _time
    while b < len(tb.lengths) and done < budget:
        n, steps = int(tb.lengths[b]), int(tb.steps[b])
        o = oracle.Oracle(oracle.D1Q2, n, 1, gamma=tb.gamma, lam=float(tb.lam[b]), omega=tb.omega,
                          bc=[("transmissive", None)] * 2, nthreads=1)
        x = (np.arange(n) + 0.5) / n
        prim = np.stack([np.where(x < 0.5, tb.left[b, k], tb.right[b, k]) for k in range(3)])
        fs = o.init(o.prim_to_cons(prim))
        _, dt = o.timed_run(fs, steps)
        t += dt
        done += n * steps
        b += 1
    v = done / t / 1e6
    out["batched_tubes_4096"] = {"workload": cfg["name"], "one_thread": {
        "value": v, "unit": UNIT, "cores": 1,
        "sample": f"the batch's first {b} tubes, whole runs, {done:.3g} updates ({t:.1f} s); a tube is one "
                  "row, which the oracle runs on one thread",
        "extrapolated_full_run_s": tb.total_updates / (v * 1e6), "extrapolated": True}}
    # 5: adjoint, forward with stored moments plus the backward sweep, at 64^2 and 512^2
    res = {"workload": "adjoint_pulses_2048 at 64 x 64 (63 steps, the FD copy) and 512 x 512 (32 steps)"}
    for n, steps in ((64, 63), (512, 32)):
        wl5, tgt = workloads.adjoint_pulses(seed=0, n=n, steps=steps)
        o = oracle.Oracle.from_workload(wl5)
        U0 = o.prim_to_cons(wl5.prim)
        t0 = _time.perf_counter()
        fsT, _ = o.run(o.init(U0), steps)
        t_fwd = _time.perf_counter() - t0
        dLdU = np.zeros_like(U0)
        dLdU[0] = (o.moments(fsT)[0] - tgt) * wl5.dx * wl5.dx
        t0 = _time.perf_counter()
        o.gradient(U0, steps, dLdU)
        t_grad = _time.perf_counter() - t0
        res[f"{n}x{n}"] = {"steps": steps, "forward_s": t_fwd, "forward_mlups": n * n * steps / t_fwd / 1e6,
                           "gradient_s": t_grad, "gradient_over_forward": t_grad / t_fwd,
                           "cores": oracle.max_threads(),
                           "note": "gradient = a forward run storing every step's moments, then the adjoint sweep"}
    out["adjoint_pulses_2048"] = res
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = workload()
    o = oracle.Oracle.from_workload(wl)
    fs = o.init(o.prim_to_cons(wl.prim))
    for _ in range(args.warmup):
        fs, _ = o.timed_run(fs, 1)
    total = 0.0
    for _ in range(args.steps):
        fs, t = o.timed_run(fs, 1)
        total += t
    value = wl.cells * args.steps / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded quadrant states)", "config": config_dict(wl, {"parallelism": parallelism(ws)}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"full {wl.nx}x{wl.ny} grid, {args.steps} steps after {args.warmup} warm-up, "
                                       "FP64 on the host cores (no L2 flush: a CPU run)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ profiling cases
#
# `python bench.py --profile CASE` runs one kernel family on a representative case, for an
# external profiler (ncu -k ... -c ...): each case holds at most about 1.5 GB on the device and
# launches its kernels a handful of times after a warm-up, and prints the wall time of its calls.

def _prof_timed(fn):
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t


def prof_step2d_f32():
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.step(1) for _ in range(wl.steps)])


def prof_step2d_f32_flushed():
    """The bench's cache state: a 256 MiB write before every call; 3 warm-up calls of two steps,
    6 timed calls of two steps (one two-step launch each), then 6 calls of one step."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def run():
        for n in [2] * 9 + [1] * 6:
            flush.fill_(1.0)
            s.step(n)
    return _prof_timed(run)


def prof_step2d_f32_flushed3():
    """The bench's headline: a 256 MiB write before every call of three steps (one launch of the
    three-step kernel); 3 warm-up calls, then 6."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def run():
        for _ in range(9):
            flush.fill_(1.0)
            s.step(3)
    return _prof_timed(run)


def prof_step2d_f16neq():
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.oblique_shock_reflection(nx=2048, ny=512, steps=10, omega=1.5)
    s = Solver.from_workload(wl, precision="f16neq")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.step(1) for _ in range(wl.steps)])


def prof_step2d_f32u_flushed():
    """The moments-only form in the bench's cache state: a 256 MiB write before every call of two steps
    (3 warm-up calls, then 6)."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=0)
    s = Solver.from_workload(wl, precision="f32u")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def run():
        for _ in range(9):
            flush.fill_(1.0)
            s.step(2)
    return _prof_timed(run)


def prof_obstacles():
    """The forward-facing step on 3072 x 1024 in FP32, 10 steps in calls of two (the two-step
    kernel with the obstacle mask)."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.forward_facing_step(nx=3072, ny=1024, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.step(2) for _ in range(wl.steps // 2)])


def prof_burgers():
    """The scalar D2Q4 lattice on case 1 of the 2-D Burgers problems, 4096 x 4096 FP32, 10 steps."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.burgers_2d(1, 4096, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.step(1) for _ in range(wl.steps)])


def prof_burgers2():
    """The same in calls of two steps (the two-steps-per-launch scalar kernel), 5 calls."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.burgers_2d(1, 4096, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.step(2) for _ in range(wl.steps // 2)])


def prof_adaptive():
    """Adaptive lambda on the 1024 x 1024 quadrant problem in FP32, 10 single adaptive steps."""
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.step_adaptive(1, 1.05) for _ in range(10)])


def prof_adjoint():
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl, target = workloads.adjoint_pulses(seed=0, n=1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    tgt = torch.from_numpy(target).float().cuda()

    def run():
        s.forward_checkpointed(12, 4)
        _, g = s.vjp_loss(tgt)
        s.backward_checkpointed(g)
    return _prof_timed(run)


def prof_batch():
    import torch
    from paper_1504_07034_gb300.solver import BatchSolver
    tb = workloads.batched_tubes(seed=0, count=512)
    steps = np.minimum(tb.steps, 96)
    s = BatchSolver.from_tubes(tb, precision="f32")
    s.tuning = (256, 4, 32)
    s.set_state(torch.from_numpy(tb.prim()).cuda())
    return _prof_timed(lambda: s.run(steps))


def prof_diagnostics():
    import torch
    from paper_1504_07034_gb300.solver import Solver
    wl = workloads.quadrant_riemann(0, 2048, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _prof_timed(lambda: [s.diagnostics() for _ in range(3)])


PROFILE_CASES = {f.__name__[len("prof_"):]: f for f in (
    prof_step2d_f32, prof_step2d_f32_flushed, prof_step2d_f32_flushed3, prof_step2d_f16neq, prof_step2d_f32u_flushed, prof_obstacles,
    prof_burgers, prof_burgers2, prof_adaptive, prof_adjoint, prof_batch, prof_diagnostics)}


# ------------------------------------------------------------------ GPU arm

def sod_measurement(Solver, stream, barrier):
    """Sod shock tube, D1Q2, 1000 cells, t = 0.2 (461 steps): wall time of the FP64 and FP32 runs (the
    single-tube context: FP32 in blocks of up to 32 steps a launch, FP64 one step a launch; and the batched
    path as a batch of one) and the density L1 against the exact Riemann solution (a latency-bound case,
    not a roofline case)."""
    import torch
    from workloads import riemann
    from paper_1504_07034_gb300.solver import BatchSolver
    wl = workloads.from_config("sod_d1q2_1000")[1]
    exact = riemann.sample(wl.gamma, wl.meta["left"], wl.meta["right"], (wl.x - 0.5) / wl.t_final)[0]
    out = {"workload": "Sod D1Q2, 1000 cells on [0, 1], t = 0.2, %d steps, lambda %.4f" % (wl.steps, wl.lam)}
    for precision in ("f64", "f32"):
        s = Solver.from_workload(wl, precision=precision, stream=stream)
        with torch.cuda.stream(stream):
            s.set_state(torch.from_numpy(wl.prim).cuda())
            s.step(wl.steps)                      # warm-up (graph capture)
            s.set_state(torch.from_numpy(wl.prim).cuda())
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a.record(stream)
            s.step(wl.steps)
            b.record(stream)
            barrier()
            rho = s.moments(torch.float64)[0].cpu().numpy()
        out[precision] = {"ms": a.elapsed_time(b), "mlups": wl.nx * wl.steps / (a.elapsed_time(b) / 1e3) / 1e6,
                          "l1_rho_vs_exact_riemann": float(np.mean(np.abs(rho - exact)))}
        s.close()
        # the same tube through the batched path, a batch of one (up to `halo` steps per launch in shared
        # memory, the single-tube arithmetic): the latency-bound run in a handful of launches
        bs = BatchSolver([wl.nx], [wl.lam], gamma=wl.gamma, omega=wl.omega, boundary="transmissive",
                         precision=precision, stream=stream)
        with torch.cuda.stream(stream):
            bs.set_state(torch.from_numpy(wl.prim).cuda())
            bs.run([wl.steps])                    # warm-up (graph capture)
            bs.set_state(torch.from_numpy(wl.prim).cuda())
            l0 = bs.launch_count
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a.record(stream)
            bs.run([wl.steps])
            b.record(stream)
            barrier()
            rho_b = bs.moments(torch.float64)[0].cpu().numpy()
            launches = bs.launch_count - l0
        out[precision]["batched_path"] = {
            "ms": a.elapsed_time(b), "mlups": wl.nx * wl.steps / (a.elapsed_time(b) / 1e3) / 1e6,
            "kernel_launches": launches, "max_abs_diff_rho_vs_single_tube_path": float(np.max(np.abs(rho_b - rho)))}
        bs.close()
    # the rest-particle model (D1Q3), which the paper reports removes the D1Q2 staircase
    wl3 = workloads.sod(1000, lattice="d1q3")
    s = Solver.from_workload(wl3, precision="f64", stream=stream, lattice="d1q3")
    with torch.cuda.stream(stream):
        s.set_state(torch.from_numpy(wl3.prim).cuda())
        s.step(wl3.steps)
        rho = s.moments(torch.float64)[0].cpu().numpy()
    s.close()
    out["d1q3_f64"] = {"steps": wl3.steps, "lambda": wl3.lam,
                       "l1_rho_vs_exact_riemann": float(np.mean(np.abs(rho - exact)))}
    return out


def oblique_measurement(Solver, stream, barrier, peak):
    """Oblique shock reflection 4096 x 1024 (512 MiB FP32 state > L2): steady MLUPS of the FP32 and the
    FP16 non-equilibrium forms, and their density L1 against the FP64 path after the full 20000 steps
    (omega = 1) and after 2000 steps at omega = 1.5 (where the non-equilibrium part is nonzero)."""
    import torch
    out = {"workload": "oblique shock reflection 4096x1024, 200 timed steps per form, CUDA-graph replay, "
                       "working set larger than L2 (no flush needed)"}
    for precision, bpl in (("f32", BYTES_PER_LUP_F32_FUSED3), ("f16neq", BYTES_PER_LUP_F16NEQ),
                           ("f32u", BYTES_PER_LUP_F32U)):
        big = workloads.from_config("oblique_shock_4096x1024", steps=216)[1]   # six 36-step graphs
        s = Solver.from_workload(big, precision=precision, stream=stream)
        with torch.cuda.stream(stream):
            s.set_state(torch.from_numpy(big.prim).cuda())
            s.step(72)                       # a 36-step graph, captured before the timing
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a.record(stream)
            s.step(big.steps)
            b.record(stream)
            barrier()
        t = a.elapsed_time(b) / 1e3
        mlups = big.cells * big.steps / t / 1e6
        out[precision] = {"value": mlups, "unit": UNIT, "algorithmic_bytes_per_lup": bpl,
                          "achieved_gbs": bpl * mlups / 1e3, "frac": bpl * mlups / 1e3 / peak}
        if precision == "f32u":                 # two steps per launch: U read and written once per two steps
            out[precision]["kernel_bytes_per_lup"] = 16
            out[precision]["kernel_frac"] = 16 * mlups / 1e3 / peak
        s.close()
    for omega, steps in ((1.0, 20000), (1.5, 2000)):
        wl = workloads.from_config("oblique_shock_4096x1024", steps=steps, omega=omega)[1]
        rho = {}
        forms = ("f64", "f32", "f16neq", "f32u") if omega == 1.0 else ("f64", "f32", "f16neq")
        with torch.cuda.stream(stream):
            for precision in forms:
                s = Solver.from_workload(wl, precision=precision, stream=stream)
                s.set_state(torch.from_numpy(wl.prim).cuda())
                if precision == "f64" and omega == 1.0:
                    # conservation against the sides' fluxes: at ten points of the run, the change of the
                    # FP64 totals over one step against that step's boundary balance
                    t_first = np.array(s.diagnostics()["totals"])
                    drift, chunk = 0.0, steps // 10
                    for _ in range(10):
                        t0 = np.array(s.diagnostics()["totals"])
                        fl = s.boundary_flux()
                        s.step(1)
                        t1 = np.array(s.diagnostics()["totals"])
                        net = np.array(fl["inflow"]) - np.array(fl["outflow"])
                        drift = max(drift, float(np.max(np.abs((t1 - t0) - net)) / np.max(np.abs(t0))))
                        s.step(chunk - 1)
                    t_last = np.array(s.diagnostics()["totals"])
                    out["fp64_flux_balance_omega1.0"] = {
                        "samples": 10, "max_rel_drift_per_step": drift,
                        "totals_change_over_run_rel": ((t_last - t_first) / np.max(np.abs(t_first))).tolist(),
                        "note": "|change of the FP64 totals over one step - (inflow - outflow)| / max_k |totals_k| "
                                "(lbrs_boundary_flux; y-momentum starts at zero, hence one scale for all fields), "
                                "max over fields and ten points of the 20000-step FP64 run"}
                else:
                    s.step(steps)
                rho[precision] = s.moments(torch.float64)[0].clone()
                if precision == "f64":
                    out_diag = s.diagnostics()
                s.close()
        stream.synchronize()
        out[f"l1_rho_vs_fp64_omega{omega}_steps{steps}"] = {
            p: float((rho[p] - rho["f64"]).abs().mean().item()) for p in forms[1:]}
        out[f"fp64_status_omega{omega}"] = out_diag["status"]
    out["value"] = out["f32"]["value"]
    out["frac"] = out["f32"]["frac"]
    return out


def obstacle_measurement(Solver, stream, barrier, peak):
    """Internal walls: the Mach 3 forward-facing step at the paper's 240 x 80 to t = 4 and the
    shock diffraction at 400 x 400 to t = 0.1561 (FP32 density L1 against FP64 over the fluid
    cells), and steady FP32 stepping of the step problem on a 6144 x 2048 grid (805 MB of
    state, larger than L2) for MLUPS and the roofline of the obstacle step kernel."""
    import torch
    out = {}
    for name, wl in (("forward_facing_step_240x80_t4", workloads.forward_facing_step()),
                     ("shock_diffraction_400x400", workloads.shock_diffraction(n=400))):
        rho = {}
        with torch.cuda.stream(stream):
            for precision in ("f64", "f32"):
                s = Solver.from_workload(wl, precision=precision, stream=stream)
                s.set_state(torch.from_numpy(wl.prim).cuda())
                s.step(wl.steps)
                rho[precision] = s.moments(torch.float64)[0].clone()
                if precision == "f64":
                    diag = s.diagnostics()
                s.close()
        stream.synchronize()
        fluid = torch.from_numpy(wl.solid == 0).cuda()
        out[name] = {"steps": wl.steps, "lambda": wl.lam,
                     "l1_rho_f32_vs_f64": float((rho["f32"] - rho["f64"])[fluid].abs().mean().item()),
                     "fp64_status": diag["status"], "fp64_min_rho": diag["min_rho"], "fp64_min_p": diag["min_p"]}
    big = workloads.forward_facing_step(nx=6144, ny=2048, steps=200)
    s = Solver.from_workload(big, precision="f32", stream=stream)
    with torch.cuda.stream(stream):
        s.set_state(torch.from_numpy(big.prim).cuda())
        s.step(64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(stream)
        s.step(big.steps)
        b.record(stream)
        barrier()
    s.close()
    t = a.elapsed_time(b) / 1e3
    mlups = big.cells * big.steps / t / 1e6
    bpl = BYTES_PER_LUP_F32_FUSED2 + 0.5
    out["steady_6144x2048_f32"] = {"value": mlups, "unit": UNIT,
                                   "kernel": "step2d_f32_fused2_tall_kernel<false, true>",
                                   "algorithmic_bytes_per_lup": bpl, "achieved_gbs": bpl * mlups / 1e3,
                                   "frac": bpl * mlups / 1e3 / peak,
                                   "note": "two steps per launch with the obstacle mask of each tile's pull "
                                           "range in shared memory: 128 B of distributions and the 1 B mask "
                                           "per cell and launch"}
    return out


def burgers_measurement(Solver, stream, barrier, peak):
    """The scalar D2Q4 lattice on the 2-D inviscid Burgers problems of Section III: density-free
    L1 distance of the FP64 and FP32 steady states (t = 3) to the exact steady solutions on the
    paper's 64 x 64 grid, and steady FP32 stepping of case 1 on 8192 x 8192 (537 MB of state,
    larger than L2) for MLUPS and the roofline (4 x 4 B read + written per update)."""
    import torch
    out = {}
    n = 64
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    for case in (1, 2):
        wl = workloads.burgers_2d(case, n)
        exact = workloads.burgers_steady_exact(case, X, Y)
        res = {"steps": wl.steps, "lambda": wl.lam}
        for precision in ("f64", "f32"):
            s = Solver.from_workload(wl, precision=precision, stream=stream)
            with torch.cuda.stream(stream):
                s.set_state(torch.from_numpy(wl.prim).cuda())
                s.step(wl.steps)
                u = s.moments(torch.float64)[0].cpu().numpy()
            s.close()
            res[f"l1_vs_exact_steady_{precision}"] = float(np.mean(np.abs(u - exact)))
        out[f"case{case}_64x64_t3"] = res
    big = workloads.burgers_2d(1, 8192, steps=200)
    s = Solver.from_workload(big, precision="f32", stream=stream)
    with torch.cuda.stream(stream):
        s.set_state(torch.from_numpy(big.prim).cuda())
        s.step(64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(stream)
        s.step(big.steps)
        b.record(stream)
        barrier()
    s.close()
    t = a.elapsed_time(b) / 1e3
    mlups = big.cells * big.steps / t / 1e6
    bpl = 32
    out["steady_8192x8192_f32"] = {"value": mlups, "unit": UNIT,
                                   "kernel": "step2ds_fused2_kernel (two steps per launch)",
                                   "algorithmic_bytes_per_lup": bpl, "achieved_gbs": bpl * mlups / 1e3,
                                   "frac": bpl * mlups / 1e3 / peak,
                                   "kernel_bytes_per_lup": bpl // 2, "kernel_frac": bpl // 2 * mlups / 1e3 / peak,
                                   "note": "frac against one read and one write of the 4 populations per step "
                                           "(32 B), kernel_frac against the kernel's own 16 B per update"}
    return out


def adaptive_measurement(Solver, stream, barrier, wl, t_final):
    """The bench workload (1024^2 quadrant Riemann) run to the configuration's final time
    with the lattice speed chosen anew every step (safety 1.05): steps taken against the
    fixed-lambda configuration, MLUPS (each step: one prep launch and one step launch with
    the fused max reduction), and the FP32 density L1 against the FP64 adaptive run."""
    import torch
    out = {"t_final": t_final, "safety": 1.05, "fixed_lambda_steps": wl.steps, "fixed_lambda": wl.lam}
    rho = {}
    for precision in ("f64", "f32"):
        s = Solver.from_workload(wl, precision=precision, stream=stream)
        with torch.cuda.stream(stream):
            s.set_state(torch.from_numpy(wl.prim).cuda())
            s.run_to_time(t_final, 1.05)                      # warm-up run
            s.set_state(torch.from_numpy(wl.prim).cuda())
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a.record(stream)
            st = s.run_to_time(t_final, 1.05, chunk=128)
            b.record(stream)
            barrier()
            rho[precision] = s.moments(torch.float64)[0].clone()
        s.close()
        sec = a.elapsed_time(b) / 1e3
        out[precision] = {"steps": st["steps"], "t_reached": st["t"], "final_lambda": st["lambda"],
                          "seconds_incl_chunk_syncs": sec, "mlups": wl.cells * st["steps"] / sec / 1e6}
    out["l1_rho_f32_vs_f64"] = float((rho["f32"] - rho["f64"]).abs().mean().item())
    return out


def batch_measurement(stream, barrier):
    """4096 shock tubes, N log-uniform in [200, 20000], to t = 0.15 in FP32 (temporal blocking)."""
    import torch
    from paper_1504_07034_gb300.solver import BatchSolver
    tb = workloads.from_config("batched_tubes_4096")[1]
    s = BatchSolver.from_tubes(tb, precision="f32", stream=stream)
    W0 = torch.from_numpy(tb.prim()).cuda()
    with torch.cuda.stream(stream):
        s.set_state(W0)
        tuning, ns = s.autotune(tb.steps)
        s.run(tb.steps)                      # warm-up: plan, graph capture and one full run
        s.set_state(W0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        l0 = s.launch_count
        a.record(stream)
        s.run(tb.steps)                      # graph replay
        b.record(stream)
        barrier()
        launches = s.launch_count - l0
        rho32 = s.moments()[0].double()
    stream.synchronize()
    t = a.elapsed_time(b) / 1e3
    lups = tb.total_updates
    s.close()
    # per-tube density L1 of FP32 against the FP64 batch (which equals the FP64 oracle per tube)
    s64 = BatchSolver.from_tubes(tb, precision="f64", stream=stream)
    with torch.cuda.stream(stream):
        s64.set_state(W0)
        s64.run(tb.steps)
        rho64 = s64.moments()[0].double()
    stream.synchronize()
    s64.close()
    diff = (rho32 - rho64).abs().cpu().numpy()
    off = np.concatenate([[0], np.cumsum(tb.lengths)])
    l1 = np.array([diff[off[b]:off[b + 1]].mean() for b in range(len(tb.lengths))])
    return {"workload": "4096 D1Q2 shock tubes, N log-uniform in [200, 20000] (sum N = %d), seeded states, "
                        "t = 0.15, FP32" % tb.total_cells,
            "l1_rho_f32_vs_f64_per_tube": {"max": float(l1.max()), "mean": float(l1.mean())},
            "lattice_updates": lups, "seconds": t, "value": lups / t / 1e6, "unit": UNIT,
            "effective_gbs_at_48_b_per_lup": 48 * lups / t / 1e9,
            "tuning": {"block": tuning[0], "cells_per_thread": tuning[1], "halo": tuning[2],
                       "autotune_ns_per_update": ns},
            "kernel_launches": launches,
            "d1q3": batch_d1q3_measurement(stream, barrier),
            "note": "temporal blocking in shared memory: up to `halo` steps per launch, so the effective "
                    "48 B/LUP bandwidth can exceed the HBM peak"}


def batch_d1q3_measurement(stream, barrier):
    """The same 4096 tubes with the rest-particle model (lambda scaled by sqrt(3/2)), FP32."""
    import torch
    from paper_1504_07034_gb300.solver import BatchSolver
    tb = workloads.batched_tubes(seed=0, count=4096, lattice="d1q3")
    s = BatchSolver.from_tubes(tb, precision="f32", stream=stream)
    W0 = torch.from_numpy(tb.prim()).cuda()
    with torch.cuda.stream(stream):
        s.set_state(W0)
        tuning, _ = s.autotune(tb.steps)
        s.run(tb.steps)
        s.set_state(W0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(stream)
        s.run(tb.steps)
        b.record(stream)
        barrier()
    s.close()
    t = a.elapsed_time(b) / 1e3
    return {"lattice_updates": tb.total_updates, "seconds": t, "value": tb.total_updates / t / 1e6, "unit": UNIT,
            "tuning": list(tuning), "effective_gbs_at_72_b_per_lup": 72 * tb.total_updates / t / 1e9}


def adjoint_measurement(Solver, stream, barrier, n=2048, steps=2000):
    """Forward (checkpointed) vs backward (recompute + adjoint) time of the density-loss gradient,
    and the FP32 gradient's error against FP64 central differences on a 64 x 64 copy."""
    import torch
    wl, target = workloads.from_config("adjoint_pulses_2048", n=n, steps=steps)[1]
    s = Solver.from_workload(wl, precision="f32", stream=stream)
    tgt = torch.from_numpy(target).float().cuda()
    W0 = torch.from_numpy(wl.prim).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(stream):
        s.set_state(W0)
        s.forward_checkpointed(64, 8)              # warm-up: graphs and kernels
        _, g = s.vjp_loss(tgt)
        s.backward_checkpointed(g)
        s.set_state(W0)
        tot0 = s.diagnostics()["totals"]
        barrier()
        ev[0].record(stream)
        s.forward_checkpointed(steps)
        ev[1].record(stream)
        tot1 = s.diagnostics()["totals"]
        loss, g = s.vjp_loss(tgt)
        ev2 = torch.cuda.Event(enable_timing=True)
        ev2.record(stream)
        grad = s.backward_checkpointed(g)
        ev[2].record(stream)
        barrier()
    t_fwd = ev[0].elapsed_time(ev[1]) / 1e3
    t_bwd = ev2.elapsed_time(ev[2]) / 1e3
    gnorm = float(grad.double().norm().item())
    s.close()
    del s
    torch.cuda.empty_cache()

    # FD check on a 64 x 64 copy run to the same final time (2000 * 64 / 2048 -> 63 steps):
    # FP32 and FP64 adjoint gradients against FP64 central differences
    fd_steps = math.ceil(steps * 64 / n)
    small, tsmall = workloads.adjoint_pulses(seed=0, n=64, steps=fd_steps)
    s32 = Solver.from_workload(small, precision="f32", stream=stream)
    s64 = Solver.from_workload(small, precision="f64", stream=stream)
    tt = torch.from_numpy(tsmall).cuda()
    with torch.cuda.stream(stream):
        s64.set_state(torch.from_numpy(small.prim).cuda())
        U0 = s64.moments(torch.float64)                # conserved initial fields
        grads = {}
        for name, sv in (("f32", s32), ("f64", s64)):
            sv.set_state(U0, primitive=False)
            sv.forward_checkpointed(fd_steps)
            _, gT = sv.vjp_loss(tt)
            grads[name] = sv.backward_checkpointed(gT).double()

        def loss64(U):
            s64.set_state(U, primitive=False)
            s64.step(fd_steps)
            return s64.vjp_loss(tt)[0]

        gen = torch.Generator(device="cpu").manual_seed(5)
        errs = {"f32": [], "f64": []}
        for _ in range(8):
            d = torch.randn(U0.shape, generator=gen, dtype=torch.float64).cuda()
            h = 1e-6 * float(U0.norm() / d.norm())
            fd = (loss64(U0 + h * d) - loss64(U0 - h * d)) / (2 * h)
            for name in errs:
                errs[name].append(abs(float((grads[name] * d).sum()) - fd) / abs(fd))
        normwise = float((grads["f32"] - grads["f64"]).norm() / grads["f64"].norm())
    stream.synchronize()
    s32.close()
    s64.close()
    drift = [abs(b - a) / abs(a) for a, b in zip(tot0, tot1)]
    return {"workload": f"{n}x{n} periodic, uniform (1, 0.5, 0.3, 1) + 8 Gaussian pulses, {steps} FP32 steps, "
                        f"density L2 loss, sqrt(T) checkpointing (segment {math.ceil(math.sqrt(steps))})",
            "conservation_drift_fp32_2000_steps": {"relative_change_of_totals": drift,
                                                    "note": "periodic grid: mass, momentum and energy totals in FP64"},
            "forward_s": t_fwd, "backward_s": t_bwd, "backward_over_forward": t_bwd / t_fwd,
            "forward_mlups": n * n * steps / t_fwd / 1e6, "loss": loss, "grad_norm": gnorm,
            "fd_check_64x64": {"steps": fd_steps, "directions": 8,
                               "f32_max_rel_err_vs_fd": max(errs["f32"]),
                               "f64_max_rel_err_vs_fd": max(errs["f64"]),
                               "f32_rel_err_vs_fd": errs["f32"], "f64_rel_err_vs_fd": errs["f64"],
                               "f32_vs_f64_gradient_normwise": normwise,
                               "reference": "FP64 GPU path central differences; 64x64 copy run to the same "
                                            "final time as the 2048^2 x 2000-step workload"}}

def run_slabs(args, ws, rank, local):
    """N > 1 GPUs: the headline grid split into N y-slabs, one per GPU (strong scaling).  Each rank
    steps its slab with the same FP32 kernels; before every three steps the ranks swap the three rows
    next to each cut (16 FP32 planes x 3 rows x 1024 cells = 192 KiB per cut and direction) with
    NCCL send/recv on the solver's stream.  Timed like the single-GPU headline: calls of two time
    steps (exchange + one launch of the two-step kernel), the L2 flushed before every call."""
    import torch
    import torch.distributed as dist
    from paper_1504_07034_gb300 import slabs
    from paper_1504_07034_gb300.solver import Solver

    wl = workload()
    j0, j1 = slabs.slab_bounds(wl.ny, ws, SLAB_HALO)[rank]
    stream = torch.cuda.Stream()
    s = Solver("d2q4", wl.nx, j1 - j0, lam=wl.lam, dx=wl.dx, bc=slabs.slab_bc(wl.bc, rank, ws, SLAB_HALO),
               gamma=wl.gamma, omega=wl.omega, precision="f32", stream=stream)
    run = slabs.DistSlab(s, rank, ws, slabs.is_periodic_y(wl.bc))
    W0 = torch.from_numpy(np.ascontiguousarray(wl.prim[:, j0:j1, :])).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()

    def tmax(x):
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    with torch.cuda.stream(stream):
        s.set_state(W0)
        run.invalidate()
        for _ in range(args.warmup):
            flush.fill_(1.0)
            run.step(SLAB_HALO)
    plan = [SLAB_HALO] * (args.steps // SLAB_HALO) + ([args.steps % SLAB_HALO] if args.steps % SLAB_HALO else [])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plan]
    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    with ClockSampler(gpu_id) as clk:
        time.sleep(0.3)
        barrier()
        l0 = s.launch_count
        with torch.cuda.stream(stream):
            for (a, b), n in zip(ev, plan):
                flush.fill_(1.0)
                a.record(stream)
                run.step(n)
                b.record(stream)
        barrier()
        launches = s.launch_count - l0
        rows = clk.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    t = tmax(sum(ms) / 1e3)
    value = wl.cells * args.steps / t / 1e6
    call_s = tmax(statistics.mean([m for m, n in zip(ms, plan) if n == SLAB_HALO] or ms) / 1e3)
    peak, peak_kind = hbm_peak()
    own_cells = wl.nx * (j1 - j0)
    achieved = 3 * BYTES_PER_LUP_F32_FUSED3 * own_cells / call_s / 1e9
    halo_bytes = sum(s.halo_size(side)[1] for side in (2, 3))

    # FP32 density L1 of the split run against the FP64 unsplit run is that of the unsplit FP32
    # run (the slabs are bit-identical to it); the diagnostics are reduced over the ranks in FP64
    with torch.cuda.stream(stream):
        s.set_state(W0)
        run.invalidate()
        run.step(CONFIG_STEPS)
    diag = run.diagnostics()

    # end to end through the public API: host fields in, 1000 steps with the exchanges, host moments out
    prim_host = torch.from_numpy(np.ascontiguousarray(wl.prim[:, j0:j1, :])).pin_memory()
    out_host = torch.empty((4, j1 - j0, wl.nx), dtype=torch.float64).pin_memory()
    e2e = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        with torch.cuda.stream(stream):
            a.record(stream)
            s.set_state(prim_host)
            run.invalidate()
            run.step(CONFIG_STEPS)
            s.moments(out=out_host)
            b.record(stream)
        barrier()
        e2e.append(tmax(a.elapsed_time(b) / 1e3))
    e2e_value = wl.cells * CONFIG_STEPS / min(e2e[1:]) / 1e6

    # the 4096 batched tubes sharded by instance (no exchange), LPT-balanced by lambda_b N_b^2
    from paper_1504_07034_gb300.shard import lpt_shards, shard_loads, tube_costs
    from paper_1504_07034_gb300.solver import BatchSolver
    tb = workloads.batched_tubes(seed=0, count=4096)
    costs = tube_costs(tb.lengths, tb.lam)
    shards = lpt_shards(costs, ws)
    mine = tb.subset(shards[rank])
    bs = BatchSolver.from_tubes(mine, precision="f32", stream=stream)
    Wt = torch.from_numpy(mine.prim()).cuda()
    with torch.cuda.stream(stream):
        bs.set_state(Wt)
        bs.autotune(mine.steps)
        bs.run(mine.steps)                      # warm-up: plan, graph capture, one full run
        bs.set_state(Wt)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with torch.cuda.stream(stream):
        a.record(stream)
        bs.run(mine.steps)
        b.record(stream)
    barrier()
    tt = tmax(a.elapsed_time(b) / 1e3)
    bs.close()
    loads = shard_loads(costs, shards)
    tubes = {"value": tb.total_updates / tt / 1e6, "unit": UNIT, "seconds": tt,
             "lattice_updates": tb.total_updates,
             "sharding": "by instance, longest-processing-time first on lambda_b N_b^2, no data exchange",
             "load_max_over_mean": max(loads) / (sum(loads) / ws)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded four-quadrant Riemann states)",
            "config": config_dict(wl, {"parallelism": parallelism(ws)}),
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "step2d_f32_fused3_kernel", "peak_kind": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": 3 * BYTES_PER_LUP_F32_FUSED3 * own_cells,
                         "note": "per rank: the slab's two-step launch plus its halo exchange per timed call "
                                 "(the slowest rank)"},
            "halo_bytes_per_exchange_per_rank": halo_bytes,
            "batched_tubes": tubes,
            "diag_after_1000_steps": {k: diag[k] for k in ("status", "min_rho", "min_p", "max_lambda_local")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(prim_host.numel() * 8) * ws,
                    "d2h_bytes_per_step": int(out_host.numel() * 8) * ws,
                    "step": "per rank: set_state(host slab rows) + 1000 steps with the exchanges + moments(host)"},
            "clocks": summarise_clocks(rows)}
    if rank == 0:
        print(json.dumps(line))
    s.close()
    return 0


def run_ours(args):
    import torch
    from paper_1504_07034_gb300.build import build as build_lib
    build_lib()
    from paper_1504_07034_gb300.solver import Solver

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        try:
            return run_slabs(args, ws, rank, local)
        finally:
            dist.destroy_process_group()

    wl = workload()
    stream = torch.cuda.Stream()
    W0 = torch.from_numpy(wl.prim).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(s, k, warm, per=1):
        """k time steps in calls of `per` steps (the last call takes the remainder), the L2
        flushed before every call; returns the per-call milliseconds and step counts."""
        plan = [per] * (k // per) + ([k % per] if k % per else [])
        with torch.cuda.stream(stream):
            for _ in range(warm):
                flush.fill_(1.0)
                s.step(per)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plan]
            barrier()
            l0 = s.launch_count
            for (a, b), n in zip(ev, plan):
                flush.fill_(1.0)
                a.record(stream)
                s.step(n)
                b.record(stream)
            barrier()
            launches = s.launch_count - l0
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, launches, plan

    # --- FP32 path: the headline ---------------------------------------------------
    s32 = Solver.from_workload(wl, precision="f32", stream=stream)
    s32.set_state(W0)
    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    with ClockSampler(gpu_id) as clk:
        time.sleep(0.3)                      # nvidia-smi up and sampling before the timed region
        t_timed = time.time()
        ms32, launches, plan = timed_steps(s32, args.steps, args.warmup, per=3)
        t_timed = time.time() - t_timed
        # the timed region lasts tens of milliseconds: keep the same flushed three-step calls
        # running (untimed) for a further 0.3 s so that the samples see the GPU under this load
        with torch.cuda.stream(stream):
            t_end = time.time() + 0.3
            while time.time() < t_end:
                for _ in range(50):
                    flush.fill_(1.0)
                    s32.step(3)
                stream.synchronize()
            s32.set_state(W0)
        rows = clk.stop()
    clocks = summarise_clocks(rows)
    clocks["window"] = (f"0.3 s before, the timed region ({1e3 * t_timed:.0f} ms wall), 0.3 s of the same "
                        "untimed calls after")
    t32 = sum(ms32) / 1e3
    if dist is not None:
        t = torch.tensor([t32], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t32 = float(t.item())
    value = ws * wl.cells * args.steps / t32 / 1e6
    # the dominant kernel: three time steps per launch, 64 B read + 64 B written per cell
    triple_ms = [m for m, n in zip(ms32, plan) if n == 3] or ms32
    avg_kernel_s = statistics.mean(triple_ms) / 1e3
    peak, peak_kind = hbm_peak()
    achieved = 3 * BYTES_PER_LUP_F32_FUSED3 * wl.cells / avg_kernel_s / 1e9
    traffic = measured_traffic(wl.cells)

    # the two-step kernel on the same flushed grid, for comparison
    ms2, _, plan2 = timed_steps(s32, min(args.steps, 200), 3, per=2)
    pair_s = statistics.mean([m for m, n in zip(ms2, plan2) if n == 2] or ms2) / 1e3
    mlups2 = wl.cells * sum(plan2) / (sum(ms2) / 1e3) / 1e6
    two_step = {"value": mlups2, "unit": UNIT, "kernel": "step2d_f32_fused2_tall_kernel<false>",
                "algorithmic_bytes_per_lup": BYTES_PER_LUP_F32_FUSED2,
                "achieved_gbs": 2 * BYTES_PER_LUP_F32_FUSED2 * wl.cells / pair_s / 1e9,
                "frac": 2 * BYTES_PER_LUP_F32_FUSED2 * wl.cells / pair_s / 1e9 / peak,
                "note": "calls of two time steps (one launch of the two-steps-per-launch kernel), the L2 "
                        "flushed before every call"}

    # the one-step kernel on the same flushed steps, for comparison
    ms1, _, _ = timed_steps(s32, min(args.steps, 200), 3, per=1)
    mlups1 = wl.cells * len(ms1) / (sum(ms1) / 1e3) / 1e6
    single_step = {"value": mlups1, "unit": UNIT, "kernel": "step2d_kernel<float>",
                   "algorithmic_bytes_per_lup": BYTES_PER_LUP_F32,
                   "achieved_gbs": BYTES_PER_LUP_F32 * mlups1 / 1e3,
                   "frac": BYTES_PER_LUP_F32 * mlups1 / 1e3 / peak,
                   "note": "one time step per launch, the L2 flushed before every step"}

    # omega = 1.5, the configuration's second relaxation rate (the full relaxation in every collision):
    # the same flushed calls of three steps, and the FP32 density error after the 1000 steps
    s15 = Solver.from_workload(wl, precision="f32", stream=stream, omega=1.5)
    s15.set_state(W0)
    ms15, _, plan15 = timed_steps(s15, min(args.steps, 201), 3, per=3)
    mlups15 = wl.cells * sum(plan15) / (sum(ms15) / 1e3) / 1e6
    # the FP64 run checks the state every step: over-relaxation without limiters can leave the physical
    # states on this problem, and the first flagged step is reported (the error is taken before it)
    r15 = Solver.from_workload(wl, precision="f64", stream=stream, omega=1.5, diag_every=1)
    with torch.cuda.stream(stream):
        r15.set_state(W0)
        r15.step(CONFIG_STEPS)
        first_bad = r15.first_bad_step()
        n15 = CONFIG_STEPS if first_bad <= 0 else first_bad - 1
        r15.set_state(W0)
        r15.step(n15)
        s15.set_state(W0)
        s15.step(n15)
        l1_15 = float((s15.moments(torch.float64)[0] - r15.moments(torch.float64)[0]).abs().mean().item())
    s15.close()
    r15.close()
    omega_1_5 = {"value": mlups15, "unit": UNIT, "omega": 1.5, "kernel": "step2d_f32_fused3_kernel",
                 "frac_per_step_128B": BYTES_PER_LUP_F32 * mlups15 / 1e3 / peak,
                 "frac_kernel_bytes": BYTES_PER_LUP_F32_FUSED3 * mlups15 / 1e3 / peak,
                 "fp64_first_flagged_step": first_bad if first_bad > 0 else None,
                 f"l1_rho_fp32_vs_fp64_after_{n15}_steps": l1_15,
                 "note": "calls of three time steps, the L2 flushed before every call, as the headline; the "
                         "FP64 run checked every step (no floors or limiters): the first step with a non-physical "
                         "cell or a local bound above lambda is reported, and the error taken before it"}

    # --- FP64 path and FP32 accuracy over the full 1000-step configuration -----------
    s64 = Solver.from_workload(wl, precision="f64", stream=stream)
    s64.set_state(W0)
    ms64, _, _ = timed_steps(s64, min(args.steps, 200), 3)
    mlups64 = wl.cells * len(ms64) / (sum(ms64) / 1e3) / 1e6
    with torch.cuda.stream(stream):
        s64.set_state(W0)
        s64.step(CONFIG_STEPS)
        s32.set_state(W0)
        s32.step(CONFIG_STEPS)
        rho64 = s64.moments(torch.float64)[0]
        rho32 = s32.moments(torch.float64)[0]
        d64 = s64.diagnostics()
    stream.synchronize()
    l1 = float((rho32 - rho64).abs().mean().item())

    # --- the omega = 1 moments-only form on the same flushed 1024^2 steps ------------
    su = Solver.from_workload(wl, precision="f32u", stream=stream)
    su.set_state(W0)
    msu, _, planu = timed_steps(su, args.steps, args.warmup, per=2)
    tu = sum(msu) / 1e3
    pair_u = [m for m, n in zip(msu, planu) if n == 2] or msu
    kernel_u_gbs = 2 * 16 * wl.cells / (statistics.mean(pair_u) / 1e3) / 1e9   # one read + one write of U per launch
    mlups_u = wl.cells * args.steps / tu / 1e6
    with torch.cuda.stream(stream):
        su.set_state(W0)
        su.step(CONFIG_STEPS)
        rho_u = su.moments(torch.float64)[0]
    stream.synchronize()
    moments_only = {"value": mlups_u, "unit": UNIT, "ms_per_step": 1e3 * tu / args.steps,
                    "kernel": "step2d_u2_kernel (two steps per launch)",
                    "algorithmic_bytes_per_lup": BYTES_PER_LUP_F32U,
                    "achieved_gbs": BYTES_PER_LUP_F32U * mlups_u / 1e3,
                    "frac": BYTES_PER_LUP_F32U * mlups_u / 1e3 / peak,
                    "kernel_bytes_per_launch": 2 * 16 * wl.cells,
                    "kernel_achieved_gbs": kernel_u_gbs, "kernel_frac": kernel_u_gbs / peak,
                    "l1_rho_vs_fp64_gpu_after_1000_steps": float((rho_u - rho64).abs().mean().item()),
                    "note": "omega = 1: the post-collision state is f^eq(U), so U alone is stored (exact "
                            "reformulation); timed like the headline, calls of two steps with the L2 flushed "
                            "before each; frac is against one read and one write of U per step (32 B), "
                            "kernel_frac against the kernel's own bytes (U read and written once per two steps)"}
    su.close()

    # --- steady stepping on a grid larger than L2: the oblique-shock case ------------
    steady = oblique_measurement(Solver, stream, barrier, peak)

    # --- Sod shock tube (1-D, latency-bound) ------------------------------------------
    sod = sod_measurement(Solver, stream, barrier)

    # --- internal walls: forward-facing step and shock diffraction ------------------
    obstacles = obstacle_measurement(Solver, stream, barrier, peak)

    # --- adaptive lambda on the bench workload, to the configuration's final time ----
    adaptive = adaptive_measurement(Solver, stream, barrier, wl, CONFIG_STEPS * wl.dx / wl.lam)

    # --- scalar D2Q4: the 2-D Burgers problems -------------------------------------
    burgers = burgers_measurement(Solver, stream, barrier, peak)

    # --- batched 1-D tubes ---------------------------------------------------------
    batched = batch_measurement(stream, barrier)

    # --- adjoint: 2048^2 periodic pulses, 2000 FP32 steps, sqrt(T) checkpointing ------
    adjoint = adjoint_measurement(Solver, stream, barrier)

    # --- end to end through the public API with host buffers -------------------------
    prim_host = torch.from_numpy(wl.prim).pin_memory()
    out_host = torch.empty((4, wl.ny, wl.nx), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for rep in range(3):
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a.record(stream)
            s32.set_state(prim_host)
            s32.step(CONFIG_STEPS)
            s32.moments(out=out_host)
            b.record(stream)
            barrier()
            e2e_ms.append(a.elapsed_time(b))
    e2e_s = min(e2e_ms[1:]) / 1e3
    e2e_value = ws * wl.cells * CONFIG_STEPS / e2e_s / 1e6

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t32 / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded four-quadrant Riemann states)",
            "config": config_dict(wl, {"parallelism": parallelism(ws)}),
            "gpu_launches": launches,
            "frac_kernel_bytes": achieved / peak,
            "frac_per_step_128B": value / (peak * 1e3 / BYTES_PER_LUP_F32),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_kernel_bytes": achieved / peak,
                         "frac_per_step_128B": value / (peak * 1e3 / BYTES_PER_LUP_F32),
                         "kernel": "step2d_f32_fused3_kernel", "peak_kind": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": 3 * BYTES_PER_LUP_F32_FUSED3 * wl.cells,
                         "algorithmic_bytes_per_lup": BYTES_PER_LUP_F32_FUSED3,
                         "timed_call": "lbrs_step(3): one launch of the three-steps-per-launch kernel",
                         "per_step_roofline": {
                             "mlups": peak * 1e3 / BYTES_PER_LUP_F32,
                             "value_over_it": value / ws / (peak * 1e3 / BYTES_PER_LUP_F32),
                             "note": "the MLUPS that the peak allows a step that reads and writes the state once "
                                     "(128 B per update); three steps per launch move 42.7 B per update, so the "
                                     "step rate can pass it"}},
            "two_step_kernel": two_step,
            "single_step_kernel": single_step,
            "omega_1_5": omega_1_5,
            "steady_large_grid": steady,
            "moments_only_omega1": moments_only,
            "adjoint": adjoint,
            "sod_1d": sod,
            "internal_walls": obstacles,
            "burgers_2d": burgers,
            "adaptive_lambda": adaptive,
            "batched_tubes": batched,
            "fp64": {"value": mlups64, "unit": UNIT, "achieved_gbs": BYTES_PER_LUP_F64 * mlups64 / 1e3,
                     "diag_after_1000_steps": {k: d64[k] for k in ("status", "min_rho", "min_p", "max_lambda_local")}},
            "accuracy": {"l1_rho_fp32_vs_fp64_gpu_after_1000_steps": l1,
                         "note": "the FP64 GPU path matches the FP64 CPU oracle to <= 1e-12 (tests)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(prim_host.numel() * 8),
                    "d2h_bytes_per_step": int(out_host.numel() * 8),
                    "step": "set_state(host) + 1000 steps + moments(host)"},
            "clocks": clocks}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(wl)
        line["cpu_baseline"]["cpu_model"] = cpu_model()
        line["cpu_baseline"]["per_config"] = oracle_per_config()
    if rank == 0:
        print(json.dumps(line))
    s32.close()
    s64.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_profile(name):
    from paper_1504_07034_gb300.build import build as build_lib
    build_lib()
    if name not in PROFILE_CASES:
        raise SystemExit(f"unknown profiling case {name}; choose from {', '.join(PROFILE_CASES)}")
    print(f"{name}: {PROFILE_CASES[name]() * 1e3:.2f} ms")
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", metavar="CASE", help="run one profiling case instead (see PROFILE_CASES)")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args.profile)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
