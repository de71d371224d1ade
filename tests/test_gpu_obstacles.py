"""GPU parity of the internal walls (lattice-aligned obstacles) through the C ABI.

Bars: FP64 GPU against the FP64 oracle to 1e-12 (normwise, distributions and moments; both
sides evaluate the same expressions in the same order, so the expected difference is zero);
FP32 against the oracle to 2e-5 normwise; solid cells carried unchanged; an all-fluid mask
gives the no-obstacle result bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()
    oracle.build()


def gpu_run(wl, precision, steps=None, solid=None):
    """solid: a mask to set in place of the workload's own (None keeps the workload's)."""
    from paper_1504_07034_gb300.solver import Solver
    s = Solver.from_workload(wl, precision=precision)
    if solid is not None:
        s.set_obstacles(solid)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(wl.steps if steps is None else steps)
    fs = s.get_distributions().double().cpu().numpy()
    U = s.moments(torch.float64).cpu().numpy()
    s.close()
    return fs, U


def oracle_run(wl, steps=None):
    o = oracle.Oracle.from_workload(wl)
    fs0 = o.init(o.prim_to_cons(wl.prim))
    fs, chk = o.run(fs0, wl.steps if steps is None else steps)
    return fs, o.moments(fs), fs0, chk


def normwise(a, b, axis):
    """Largest |a - b| relative to the largest |b|, taken per conserved field (axis: the field
    axis of the arrays; a field that is zero throughout is scaled by the largest of all)."""
    a, b = np.moveaxis(np.asarray(a), axis, 0), np.moveaxis(np.asarray(b), axis, 0)
    glob = float(np.max(np.abs(b)))
    return max(float(np.max(np.abs(a[k] - b[k]))) / (float(np.max(np.abs(b[k]))) or glob) for k in range(b.shape[0]))


def test_f64_forward_facing_step_matches_oracle():
    """The paper's 240 x 80 Mach 3 step to t = 4 (2119 steps; graph replay)."""
    wl = W.forward_facing_step()
    fr, Ur, fs0, _ = oracle_run(wl)
    fs, U = gpu_run(wl, "f64")
    assert normwise(fs, fr, 1) <= F64_TOL
    assert normwise(U, Ur, 0) <= F64_TOL
    solid = wl.solid == 1
    assert np.array_equal(fs[:, :, solid], fs0[:, :, solid])


def test_f64_shock_diffraction_matches_oracle():
    wl = W.shock_diffraction(n=200)
    fr, Ur, _, _ = oracle_run(wl)
    fs, U = gpu_run(wl, "f64")
    assert normwise(fs, fr, 1) <= F64_TOL
    assert normwise(U, Ur, 0) <= F64_TOL


P = ("periodic", None)
T = ("transmissive", None)
WALL = ("wall", None)
BC_SETS = {
    "periodic": [P, P, P, P],
    "walls_periodic_x": [P, P, WALL, WALL],
    "transmissive": [T, T, T, T],
    "mixed": [("dirichlet", (1.1, 0.3, 0.0, 1.0)), T, WALL, ("dirichlet", (0.9, 0.2, -0.1, 0.8))],
}


def random_obstacle_case(nx, ny, bcname, omega, seed, steps=60):
    """Smooth state, a few random rectangles (kept only if the oracle accepts the geometry)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / max(nx, ny)
    y = (np.arange(ny) + 0.5) / max(nx, ny)
    X, Y = np.meshgrid(x, y)
    prim = np.array([1 + 0.15 * np.sin(6 * X + 1) * np.cos(5 * Y), 0.3 + 0.1 * np.cos(7 * Y),
                     -0.1 + 0.1 * np.sin(4 * X), 1 + 0.1 * np.cos(5 * (X + Y))])
    bc = BC_SETS[bcname]
    if bc[2] == WALL:
        prim[2, 0] = 0.0
    if bc[3] == WALL:
        prim[2, -1] = 0.0
    for _ in range(200):
        solid = np.zeros((ny, nx), np.uint8)
        for _ in range(rng.integers(1, 5)):
            w, h = rng.integers(1, max(2, nx // 3)), rng.integers(1, max(2, ny // 3))
            i0, j0 = rng.integers(0, nx - w + 1), rng.integers(0, ny - h + 1)
            solid[j0:j0 + h, i0:i0 + w] = 1
        try:
            oracle.Oracle(oracle.D2Q4, nx, ny, lam=4.0, omega=omega, bc=bc, solid=solid)
        except ValueError:
            continue
        return W.Workload2D(f"obstacles_{bcname}", nx, ny, 1.0 / max(nx, ny), 0.0, 0.0, prim, bc, 4.0, omega,
                            steps, solid=solid)
    raise RuntimeError("no valid geometry drawn")


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
@pytest.mark.parametrize("shape", [(64, 40), (37, 29), (130, 18)])
@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_f64_random_obstacles_match_oracle(bcname, shape, omega):
    seed = 100 * sorted(BC_SETS).index(bcname) + shape[0] + int(10 * omega)
    wl = random_obstacle_case(*shape, bcname, omega, seed=seed)
    fr, Ur, _, _ = oracle_run(wl)
    fs, U = gpu_run(wl, "f64")
    assert normwise(fs, fr, 1) <= F64_TOL
    assert normwise(U, Ur, 0) <= F64_TOL


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
def test_f32_random_obstacles_close_to_oracle(bcname):
    wl = random_obstacle_case(96, 48, bcname, 1.3, seed=7, steps=80)
    _, Ur, _, _ = oracle_run(wl)
    _, U = gpu_run(wl, "f32")
    err = np.max(np.abs(U - Ur), axis=(1, 2)) / np.max(np.abs(Ur))
    assert np.all(err <= 2e-5), err


def test_f32_forward_facing_step_close_to_oracle():
    wl = W.forward_facing_step()
    _, Ur, _, _ = oracle_run(wl)
    _, U = gpu_run(wl, "f32")
    fluid = wl.solid == 0
    l1 = float(np.mean(np.abs(U[0][fluid] - Ur[0][fluid])))
    assert l1 <= 1e-5, l1


_FUSE_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import workloads as W
from test_gpu_obstacles import random_obstacle_case
from paper_1504_07034_gb300.solver import Solver
cases = [W.forward_facing_step(), W.shock_diffraction(n=200)]
for k, (nx, ny) in enumerate(((64, 40), (132, 18), (36, 29), (96, 48), (37, 29))):
    for bcname in ("periodic", "walls_periodic_x", "transmissive", "mixed"):
        cases.append(random_obstacle_case(nx, ny, bcname, (1.0, 1.6)[k % 2], seed=11 * k + len(bcname), steps=0))
out = []
for wl in cases:
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(51)
    out.append(s.get_distributions().cpu().numpy().ravel())
    out.append(s.step_record(5).cpu().numpy().ravel())
    out.append(s.get_distributions().cpu().numpy().ravel())
    s.close()
np.save(sys.argv[2], np.concatenate(out))
"""


def test_f32_two_step_kernel_with_walls_equals_single_steps(tmp_path):
    """The two-steps-per-launch kernel with internal walls (tensor copies where nx % 4 == 0;
    the mask of each tile's pull range in shared memory) against one-step launches, bit for
    bit: both run the same per-cell code (pull, mirror rule, collision).  Random rectangles
    under every boundary set, ragged tiles, the forward-facing step and the shock
    diffraction; 51 steps (a graph, pairs and a single step), then 5 recording steps."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fuse_walls.py"
    script.write_text(_FUSE_SCRIPT)
    res = {}
    for fuse in ("0", "1"):
        out = tmp_path / f"f{fuse}.npy"
        subprocess.run([sys.executable, str(script), root, str(out)], check=True,
                       env=dict(os.environ, LBRS_F32_FUSE=fuse), timeout=600)
        res[fuse] = np.load(out)
    assert np.array_equal(res["1"], res["0"]), np.max(np.abs(res["1"] - res["0"]))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_all_fluid_mask_equals_no_obstacles(precision):
    wl = random_obstacle_case(70, 40, "mixed", 1.2, seed=3, steps=70)
    wl.solid = None
    f_plain, _ = gpu_run(wl, precision)
    f_mask, _ = gpu_run(wl, precision, solid=np.zeros((wl.ny, wl.nx), np.uint8))
    assert np.array_equal(f_plain, f_mask)


def test_obstacle_errors():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    # a fluid channel one cell wide
    s = Solver.from_workload(W.uniform_2d(16, 12), precision="f64")
    bad = np.zeros((s.ny, s.nx), np.uint8)
    bad[: s.ny // 2 - 1] = 1
    bad[s.ny // 2:] = 1
    with pytest.raises(abi.LbrsError) as e:
        s.set_obstacles(bad)
    assert e.value.status == abi.LBRS_EINVAL
    s.close()
    # storage forms and lattices without internal walls
    s = Solver.from_workload(W.oblique_shock_reflection(nx=64, ny=16, steps=0), precision="f16neq")
    with pytest.raises(abi.LbrsError):
        s.set_obstacles(np.zeros((16, 64), np.uint8))
    s.close()
    s = Solver.from_workload(W.sod(100), precision="f64")
    with pytest.raises((abi.LbrsError, ValueError)):
        s.set_obstacles(np.zeros((1, 100), np.uint8))
    s.close()
    # the adjoint does not cover internal walls
    wlp, _ = W.adjoint_pulses(seed=0, n=32, steps=0)
    s = Solver.from_workload(wlp, precision="f32")
    m = np.zeros((32, 32), np.uint8)
    m[10:14, 10:14] = 1
    s.set_obstacles(m)
    s.set_state(torch.from_numpy(wlp.prim).cuda())
    with pytest.raises(abi.LbrsError):
        s.forward_checkpointed(10, 3)
    # removing the walls
    s.set_obstacles(None)
    s.forward_checkpointed(10, 3)
    s.close()
