"""The omega = 1 moments-only form (LBRS_F32U) and the shared-memory tile kernel.

At omega = 1 the post-collision state is f^eq(U), so storing U alone is an exact
reformulation: the form must agree with the FP32 distribution-storing path up
to FP32 rounding, and with the FP64 oracle within the FP32 bar, on every
boundary kind and on tiles cut by the domain edge (nx, ny not multiples of the
32 x 16 tile).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()
    oracle.build()


def run(wl, precision, steps=None):
    from paper_1504_07034_gb300.solver import Solver
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(wl.steps if steps is None else steps)
    U = s.moments().cpu().numpy()
    s.close()
    return U


@pytest.mark.parametrize("bc", ["transmissive", "periodic", "dirichlet_wall", "walls_periodic_x", "mixed"])
@pytest.mark.parametrize("shape", [(160, 96), (37, 29), (1, 9), (33, 1), (70, 18)])
def test_f32u_equals_f32_path_at_omega1(bc, shape):
    from test_gpu_parity import small_case
    nx, ny = shape
    if bc in ("periodic", "walls_periodic_x"):
        nx += nx % 2
        ny += ny % 2
    if "wall" in bc and ny < 2:
        ny = 2
    wl = small_case(nx, ny, bc, 1.0, steps=80)
    Uu = run(wl, "f32u")
    U32 = run(wl, "f32")
    ref = run(wl, "f64")
    scale = np.abs(ref).max()
    assert np.max(np.abs(Uu - U32)) <= 1e-5 * scale
    assert np.max(np.abs(Uu - ref)) <= 2e-5 * scale


def test_f32u_full_size_quadrant_against_oracle():
    wl = W.quadrant_riemann(0, 1024, steps=1000)
    o = oracle.Oracle.from_workload(wl)
    fs, _ = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps)
    ref = o.moments(fs)
    U = run(wl, "f32u")
    l1 = float(np.mean(np.abs(U[0] - ref[0])))
    print(f"quadrant 1024^2 x 1000, moments-only FP32: density L1 vs FP64 oracle {l1:.2e}")
    assert l1 <= 1e-5


def test_f32u_needs_omega_one():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl = W.quadrant_riemann(0, 16, omega=1.5)
    with pytest.raises(abi.LbrsError) as e:
        Solver.from_workload(wl, precision="f32u")
    assert "omega" in str(e.value)


def test_f32u_checkpoint_and_diagnostics():
    from paper_1504_07034_gb300.solver import Solver
    wl = W.oblique_shock_reflection(nx=256, ny=64, steps=0)
    a = Solver.from_workload(wl, precision="f32u")
    a.set_state(torch.from_numpy(wl.prim).cuda())
    a.step(40)
    raw = a.raw_state().clone()
    a.step(30)
    end = a.moments()
    b = Solver.from_workload(wl, precision="f32u")
    b.set_raw_state(raw, step=40)
    b.step(30)
    assert torch.equal(b.moments(), end)
    d = a.diagnostics()
    assert d["status"] == "LBRS_OK"
    assert d["min_rho"] == pytest.approx(float(end[0].min()), rel=1e-6)
    a.close()
    b.close()


_FUSE_SCRIPT = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
sys.path.insert(0, sys.argv[1] + "/tests")
from test_gpu_parity import small_case
from paper_1504_07034_gb300.solver import Solver
out = []
for bc in ("transmissive", "periodic", "dirichlet_wall", "walls_periodic_x", "mixed"):
    for nx, ny in ((160, 96), (37, 29), (2, 2), (1, 9), (33, 1), (70, 18), (66, 34)):
        if bc in ("periodic", "walls_periodic_x"):
            nx += nx % 2
            ny += ny % 2
        if "wall" in bc and ny < 2:
            ny = 2
        wl = small_case(nx, ny, bc, 1.0, steps=51)
        s = Solver.from_workload(wl, precision="f32u")
        s.set_state(torch.from_numpy(wl.prim).cuda())
        s.step(51)                    # a 32-step graph, then 9 two-step launches and one single step
        out.append(s.raw_state().cpu().numpy().copy())
        s.step(3)
        out.append(s.raw_state().cpu().numpy().copy())
        s.close()
np.save(sys.argv[2], np.concatenate(out))
"""


def test_f32u_two_step_kernel_equals_single_steps(tmp_path):
    """The two-steps-per-launch kernel of the moments-only form forms every value with the
    single-step kernel's arithmetic (window rebuilt twice, wall relations, boundary
    resolution), so the states must agree bit for bit: every boundary set, ragged tiles,
    grids narrower than the window (one-cell and two-cell periodic axes)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fuse.py"
    script.write_text(_FUSE_SCRIPT)
    res = {}
    for fuse in ("0", "1"):
        out = tmp_path / f"fuse{fuse}.npy"
        env = dict(os.environ, LBRS_F32U_FUSE=fuse)
        subprocess.run([sys.executable, str(script), root, str(out)], check=True, env=env, timeout=300)
        res[fuse] = np.load(out)
    assert np.array_equal(res["0"], res["1"])
