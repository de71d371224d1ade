"""FP32 1-D steps in blocks: a tube of one through the batched tubes' temporal-blocking kernel.

An FP32 D1Q2 or D1Q3 context whose ends are both transmissive or both periodic advances up to 32
steps per launch in shared memory (tiles of 960 cells), with the per-cell arithmetic of the
one-step kernel.  The state after any number of steps must equal one step per launch
(LBRS_1D_BLOCKED=0) bit for bit: tube lengths around the tile size, step counts around the 32-step
block, both lattices, both end conditions, omega = 1 and 1.5.  The Sod run is also held to the
FP64 oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1504_07034_gb300.solver import Solver
rng = np.random.default_rng(3)
out, launches = [], []
for lattice in ("d1q2", "d1q3"):
    for ends in ("transmissive", "periodic"):
        for omega in (1.0, 1.5):
            for nx in (1, 2, 5, 959, 960, 961, 1000, 3001):
                if ends == "periodic" and nx % 2:
                    nx += 1
                x = (np.arange(nx) + 0.5) / nx
                rho = np.where(x < 0.5, 1.0, 0.125) + 0.05 * rng.random(nx)
                u = 0.2 * rng.standard_normal(nx)
                p = np.where(x < 0.5, 1.0, 0.1) + 0.05 * rng.random(nx)
                lam = 3.5 * (1.22 if lattice == "d1q3" else 1.0)
                s = Solver(lattice, nx, 1, lam=lam, dx=1.0 / nx, bc=[(ends, None)] * 2, omega=omega,
                           precision="f32")
                s.set_state(torch.from_numpy(np.stack([rho, u, p])).cuda())
                for n in (1, 31, 32, 33, 100):
                    l0 = s.launch_count
                    s.step(n)
                    torch.cuda.synchronize()
                    launches.append(s.launch_count - l0)
                    out.append(s.get_distributions().cpu().numpy().ravel())
                s.close()
np.save(sys.argv[2], np.concatenate(out))
np.save(sys.argv[3], np.array(launches))
"""


def test_blocked_1d_steps_equal_single_steps(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "oned.py"
    script.write_text(_SCRIPT)
    res, nl = {}, {}
    for name, env_add in (("blocked", {}), ("single", {"LBRS_1D_BLOCKED": "0"})):
        out, lout = tmp_path / f"{name}.npy", tmp_path / f"{name}_launches.npy"
        subprocess.run([sys.executable, str(script), root, str(out), str(lout)], check=True,
                       env=dict(os.environ, **env_add), timeout=600)
        res[name], nl[name] = np.load(out), np.load(lout)
    assert np.all(np.isfinite(res["single"]))
    assert np.array_equal(res["blocked"], res["single"]), np.max(np.abs(res["blocked"] - res["single"]))
    # blocks of up to 32 steps: 1, 31, 32, 33 and 100 steps take 1, 1, 1, 2 and 4 launches
    assert np.array_equal(nl["blocked"], np.tile([1, 1, 1, 2, 4], len(nl["blocked"]) // 5))
    assert np.array_equal(nl["single"], np.tile([1, 31, 32, 33, 100], len(nl["single"]) // 5))


def test_blocked_sod_close_to_oracle():
    """The Sod configuration (1000 cells, 461 steps) in FP32 blocks against the FP64 oracle."""
    from paper_1504_07034_gb300.solver import Solver
    wl = W.sod(1000)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    l0 = s.launch_count
    s.step(wl.steps)
    assert s.launch_count - l0 == (wl.steps + 31) // 32
    U = s.moments(torch.float64).cpu().numpy()
    s.close()
    o = oracle.Oracle.from_workload(wl)
    fs, _ = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps)
    ref = o.moments(fs)
    assert np.mean(np.abs(U[0] - ref[0])) <= 1e-6
