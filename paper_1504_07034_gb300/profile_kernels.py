"""Run one kernel family of the library on a representative case, for an external profiler.

    python -m paper_1504_07034_gb300.profile_kernels CASE

CASE: step2d_f32 | step2d_f32_flushed | step2d_f16neq | obstacles | adjoint |
batch | diagnostics.  Each case
holds at most about 1.5 GB on the device and launches its kernels a handful
of times after a warm-up, so that a profiler capture (`ncu -k ... -c ...`)
stays small.  It prints one line per case with the wall time of its kernels.
"""
from __future__ import annotations

import sys
import time

import numpy as np
import torch

import workloads


def _timed(fn):
    torch.cuda.synchronize()
    t = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t


def step2d_f32():
    from .solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _timed(lambda: [s.step(1) for _ in range(wl.steps)])


def step2d_f32_flushed():
    """The bench's cache state: a 256 MiB write before every call; 3 warm-up calls of two steps,
    6 timed calls of two steps (one two-step launch each), then 6 calls of one step."""
    from .solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def run():
        for n in [2] * 9 + [1] * 6:
            flush.fill_(1.0)
            s.step(n)
    return _timed(run)


def step2d_f16neq():
    from .solver import Solver
    wl = workloads.oblique_shock_reflection(nx=2048, ny=512, steps=10, omega=1.5)
    s = Solver.from_workload(wl, precision="f16neq")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _timed(lambda: [s.step(1) for _ in range(wl.steps)])


def obstacles():
    """The forward-facing step on 3072 x 1024 in FP32, 10 steps in calls of two (the two-step
    kernel with the obstacle mask)."""
    from .solver import Solver
    wl = workloads.forward_facing_step(nx=3072, ny=1024, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _timed(lambda: [s.step(2) for _ in range(wl.steps // 2)])


def burgers():
    """The scalar D2Q4 lattice on case 1 of the 2-D Burgers problems, 4096 x 4096 FP32, 10 steps."""
    from .solver import Solver
    wl = workloads.burgers_2d(1, 4096, steps=10)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _timed(lambda: [s.step(1) for _ in range(wl.steps)])


def adaptive():
    """Adaptive lambda on the 1024 x 1024 quadrant problem in FP32, 10 single adaptive steps."""
    from .solver import Solver
    wl = workloads.quadrant_riemann(0, 1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _timed(lambda: [s.step_adaptive(1, 1.05) for _ in range(10)])


def adjoint():
    from .solver import Solver
    wl, target = workloads.adjoint_pulses(seed=0, n=1024, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    tgt = torch.from_numpy(target).float().cuda()

    def run():
        s.forward_checkpointed(12, 4)
        _, g = s.vjp_loss(tgt)
        s.backward_checkpointed(g)
    return _timed(run)


def batch():
    from .solver import BatchSolver
    tb = workloads.batched_tubes(seed=0, count=512)
    steps = np.minimum(tb.steps, 96)
    s = BatchSolver.from_tubes(tb, precision="f32")
    s.tuning = (256, 4, 32)
    s.set_state(torch.from_numpy(tb.prim()).cuda())
    return _timed(lambda: s.run(steps))


def diagnostics():
    from .solver import Solver
    wl = workloads.quadrant_riemann(0, 2048, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    return _timed(lambda: [s.diagnostics() for _ in range(3)])


CASES = {f.__name__: f for f in (step2d_f32, step2d_f32_flushed, step2d_f16neq, obstacles, burgers, adaptive,
                                 adjoint, batch, diagnostics)}


def main(argv):
    from .build import build
    build()
    names = argv[1:] or list(CASES)
    for name in names:
        if name not in CASES:
            raise SystemExit(f"unknown case {name}; choose from {', '.join(CASES)}")
        print(f"{name}: {CASES[name]() * 1e3:.2f} ms")


if __name__ == "__main__":
    main(sys.argv)
