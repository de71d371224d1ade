"""The bounds-checked build (liblbrs_debug.so, -DLBRS_DEBUG): the library's check of its own
index arithmetic where no memory sanitizer runs.

A matrix of degenerate and ragged grids (1 x 1 to several tiles), every boundary set, the FP64,
FP32, FP16 non-equilibrium and moments-only forms, the two-steps-per-launch kernel (with and
without internal walls), graph replay, recording steps, the scalar lattice, D1Q2 / D1Q3 tubes,
batched tubes of ragged lengths, adaptive steps and the checkpointed adjoint runs through the
bounds-checked library in a child process: no checked index may leave its buffer
(lbrs_debug_check after every case), and the results must equal the release library's: bit for
bit where the arithmetic is compiled without contraction (FP64), to 1e-5 of the field's scale
otherwise (the checks change the code around the arithmetic, and with it where the compiler may
fuse a multiply and an add).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import ctypes
import sys

import numpy as np
import torch

sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import workloads as W
from paper_1504_07034_gb300 import abi
from paper_1504_07034_gb300.solver import BatchSolver, Solver
from test_gpu_obstacles import random_obstacle_case

lib = abi.load()
out, names, records = [], [], []


def check(name):
    torch.cuda.synchronize()
    w = ctypes.c_uint64(0)
    lib.lbrs_debug_check(ctypes.byref(w))
    if w.value:
        records.append((name, int(w.value) >> 40, int(w.value) & ((1 << 40) - 1)))


def keep(name, t):
    out.append(t.detach().double().cpu().numpy().ravel())
    names.append(name)


T = ("transmissive", None)
P = ("periodic", None)
WL = ("wall", None)
D = [("dirichlet", (1.0, 0.5, 0.1, 1.0)), ("dirichlet", (0.8, -0.2, 0.0, 0.9))]
BCS = {"transmissive": [T] * 4, "periodic": [P] * 4, "mixed": [D[0], T, WL, D[1]], "walls_x_periodic": [P, P, WL, WL]}
base = W.quadrant_riemann(1, 64, steps=0)
for precision in ("f64", "f32", "f16neq", "f32u"):
    for bname, bc in BCS.items():
        for nx, ny in ((1, 1), (1, 9), (33, 1), (5, 3), (37, 29), (36, 20), (66, 17), (132, 18), (98, 66)):
            if bc[0] == P and nx % 2:
                nx += 1
            if bc[2] == P and ny % 2:
                ny += 1
            if WL in (bc[2], bc[3]):
                ny = max(ny, 2)
            prim = np.ascontiguousarray(np.tile(base.prim, (1, 2, 4))[:, :ny, :nx])
            if bc[2] == WL:
                prim[2, 0, :] = 0.0
            if bc[3] == WL:
                prim[2, -1, :] = 0.0
            omega = 1.0 if precision == "f32u" else 1.3
            s = Solver("d2q4", nx, ny, lam=1.6 * base.lam, dx=1.0 / 64, bc=bc, omega=omega, precision=precision)
            s.set_state(torch.from_numpy(prim).cuda())
            s.step(13)
            name = f"{precision}-{bname}-{nx}x{ny}"
            keep(name, s.get_distributions() if precision in ("f64", "f32") else s.moments())
            if precision in ("f64", "f32"):
                keep(name + "-record", s.step_record(5))
            s.close()
            check(name)
# graph replay of the two-step kernel on a grid of several tiles
s = Solver.from_workload(W.quadrant_riemann(2, 96, steps=0), precision="f32")
s.set_state(torch.from_numpy(W.quadrant_riemann(2, 96, steps=0).prim).cuda())
s.step(70)
keep("graph-f32", s.get_distributions())
s.close()
check("graph-f32")
# internal walls, both precisions
for k, (nx, ny) in enumerate(((36, 29), (132, 18), (64, 40))):
    for bname in ("periodic", "mixed", "walls_periodic_x"):
        wl = random_obstacle_case(nx, ny, bname, 1.2, seed=7 * k + len(bname), steps=0)
        for precision in ("f64", "f32"):
            s = Solver.from_workload(wl, precision=precision)
            s.set_state(torch.from_numpy(wl.prim).cuda())
            s.step(11)
            keep(f"walls-{precision}-{bname}-{nx}x{ny}", s.get_distributions())
            s.close()
            check(f"walls-{precision}-{bname}-{nx}x{ny}")
# scalar lattice
for precision in ("f64", "f32"):
    wl = W.burgers_2d(2, 40)
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(21)
    keep(f"burgers-{precision}", s.get_distributions())
    s.close()
    check(f"burgers-{precision}")
# tubes
for lattice in ("d1q2", "d1q3"):
    for n in (1, 2, 37):
        for precision in ("f64", "f32"):
            wl = W.sod(n, lattice=lattice)
            s = Solver.from_workload(wl, precision=precision, lattice=lattice)
            s.set_state(torch.from_numpy(wl.prim).cuda())
            s.step(9)
            keep(f"tube-{lattice}-{precision}-{n}", s.get_distributions())
            s.close()
            check(f"tube-{lattice}-{precision}-{n}")
    tb = W.batched_tubes(seed=3, count=19, n_min=1, n_max=600, t_final=0.15, lattice=lattice)
    steps = np.random.default_rng(3).integers(0, 200, size=19)
    for precision in ("f64", "f32"):
        b = BatchSolver(tb.lengths, tb.lam, gamma=tb.gamma, omega=tb.omega, precision=precision, lattice=lattice)
        b.set_state(torch.from_numpy(tb.prim()).cuda())
        b.run(steps)
        keep(f"batch-{lattice}-{precision}", b.moments())
        b.close()
        check(f"batch-{lattice}-{precision}")
# adaptive steps
for precision in ("f64", "f32"):
    wl = W.oblique_shock_reflection(nx=96, ny=24, steps=0)
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step_adaptive(9, 1.1)
    keep(f"adaptive-{precision}", s.get_distributions())
    s.close()
    check(f"adaptive-{precision}")
# checkpointed adjoint on a periodic grid
for precision in ("f64", "f32"):
    wl, target = W.adjoint_pulses(seed=0, n=36, steps=0, width=0.1, pulses=3)
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.forward_checkpointed(23, 5)
    _, gT = s.vjp_loss(torch.from_numpy(target).cuda())
    keep(f"adjoint-{precision}", s.backward_checkpointed(gT))
    s.close()
    check(f"adjoint-{precision}")
np.savez(sys.argv[2], names=np.array(names), debug=lib.lbrs_debug_build(),
         records=np.array([f"{n}: site {s}, index {i}" for n, s, i in records]),
         **{f"a{k}": v for k, v in enumerate(out)})
"""


def _run(tmp_path, lib_path, tag):
    script = tmp_path / "cases.py"
    script.write_text(_SCRIPT)
    out = tmp_path / f"{tag}.npz"
    env = dict(os.environ)
    if lib_path is not None:
        env["LBRS_LIBRARY"] = str(lib_path)
    subprocess.run([sys.executable, str(script), ROOT, str(out)], check=True, env=env, timeout=900)
    return np.load(out)


def test_bounds_checked_build_stays_in_bounds_and_matches_release(tmp_path):
    from paper_1504_07034_gb300.build import build
    build()
    debug_lib = build(debug=True)
    dbg = _run(tmp_path, debug_lib, "debug")
    rel = _run(tmp_path, None, "release")
    assert int(dbg["debug"]) == 1 and int(rel["debug"]) == 0
    assert len(dbg["records"]) == 0, list(dbg["records"])
    assert list(dbg["names"]) == list(rel["names"])
    for k, name in enumerate(rel["names"]):
        a, b = dbg[f"a{k}"], rel[f"a{k}"]
        assert not np.isnan(b).any(), name
        if "f64" in name:
            assert np.array_equal(a, b), name
        else:
            assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(b)), name
