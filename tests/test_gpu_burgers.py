"""GPU parity of the scalar D2Q4 lattice (the 2-D inviscid Burgers law of Section III)
through the C ABI.

Bars: FP64 GPU against the FP64 oracle to 1e-12 normwise (distributions and moments; the same
expressions in the same order); FP32 against the oracle to 2e-5 normwise; the diagnostics'
totals, min u and bound |u| + 1 against the moments.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
P = ("periodic", None)
T = ("transmissive", None)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()
    oracle.build()


def gpu_run(wl, precision, steps=None):
    from paper_1504_07034_gb300.solver import Solver
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(wl.steps if steps is None else steps)
    fs = s.get_distributions().double().cpu().numpy()
    U = s.moments(torch.float64).cpu().numpy()
    d = s.diagnostics()
    s.close()
    return fs, U, d


def oracle_run(wl, steps=None):
    o = oracle.Oracle.from_workload(wl)
    fs, chk = o.run(o.init(wl.prim), wl.steps if steps is None else steps)
    return fs, o.moments(fs)


def normwise(a, b, axis):
    """Largest |a - b| relative to the largest |b|, taken per conserved field (axis: the field
    axis of the arrays; a field that is zero throughout is scaled by the largest of all)."""
    a, b = np.moveaxis(np.asarray(a), axis, 0), np.moveaxis(np.asarray(b), axis, 0)
    glob = float(np.max(np.abs(b)))
    return max(float(np.max(np.abs(a[k] - b[k]))) / (float(np.max(np.abs(b[k]))) or glob) for k in range(b.shape[0]))


@pytest.mark.parametrize("case", [1, 2])
@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_f64_section3_problems_match_oracle(case, omega):
    wl = W.burgers_2d(case, 64, omega=omega)
    fr, Ur = oracle_run(wl)
    fs, U, _ = gpu_run(wl, "f64")
    assert normwise(fs, fr, 1) <= F64_TOL
    assert normwise(U, Ur, 0) <= F64_TOL


def scalar_case(nx, ny, bc, omega, steps, seed=0):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / max(nx, ny)
    y = (np.arange(ny) + 0.5) / max(nx, ny)
    X, Y = np.meshgrid(x, y)
    a = rng.uniform(0.2, 0.6, 3)
    u = a[0] * np.sin(7 * X + 1) + a[1] * np.cos(5 * Y) - a[2] * X * Y
    return W.Workload2D("scalar", nx, ny, 1.0 / max(nx, ny), 0.0, 0.0, u[None].copy(), bc, 3.0, omega, steps,
                        law="burgers")


BC_SETS = {
    "periodic": [P, P, P, P],
    "transmissive": [T, T, T, T],
    "profiles": [("dirichlet", (0.4, -0.3, 0, 0)), ("dirichlet", (-0.2, 0.5, 0, 0)),
                 ("dirichlet", (0.6, -1.0, 0, 0)), ("dirichlet", (-0.3, 0.2, 0, 0))],
    "mixed": [P, P, ("dirichlet", (0.5, -0.8, 0, 0)), T],
}


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
@pytest.mark.parametrize("shape", [(37, 29), (130, 18), (2, 3), (1, 1)])
def test_f64_scalar_boundaries_and_shapes(bcname, shape):
    wl = scalar_case(*shape, BC_SETS[bcname], 1.3, 70)
    fr, Ur = oracle_run(wl)
    fs, U, _ = gpu_run(wl, "f64")
    assert normwise(fs, fr, 1) <= F64_TOL
    assert normwise(U, Ur, 0) <= F64_TOL


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
def test_f32_close_to_oracle(bcname):
    wl = scalar_case(96, 40, BC_SETS[bcname], 1.0, 120, seed=3)
    _, Ur = oracle_run(wl)
    _, U, _ = gpu_run(wl, "f32")
    assert normwise(U, Ur, 0) <= 2e-5


def test_diagnostics_of_the_scalar():
    wl = W.burgers_2d(2, 48)
    _, U, d = gpu_run(wl, "f64")
    u = U[0]
    assert d["status"] == "LBRS_OK"
    assert d["totals"][0] == pytest.approx(u.sum() * wl.dx * wl.dx, rel=1e-12)
    assert d["min_rho"] == pytest.approx(u.min(), rel=1e-12)
    assert d["max_lambda_local"] == pytest.approx(np.abs(u).max() + 1.0, rel=1e-12)


def test_scalar_lattice_rejections():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl = W.burgers_2d(1, 32)
    for precision in ("f16neq", "f32u"):
        with pytest.raises(abi.LbrsError):
            Solver.from_workload(wl, precision=precision)
    with pytest.raises(abi.LbrsError):
        Solver("d2q4s", 32, 32, lam=3.0, dx=1 / 32, bc=[P, P, ("wall", None), ("wall", None)], precision="f64")
    s = Solver.from_workload(W.burgers_2d(1, 32, t_final=0.1), precision="f32")
    with pytest.raises(abi.LbrsError):
        s.set_obstacles(np.zeros((32, 32), np.uint8))
    s.set_state(torch.from_numpy(wl.prim).cuda())
    with pytest.raises(abi.LbrsError):
        s.forward_checkpointed(4, 2)
    s.close()


_FUSE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from test_gpu_burgers import BC_SETS, scalar_case
from paper_1504_07034_gb300.solver import Solver
out = []
for bcname in sorted(BC_SETS):
    for shape in ((37, 29), (130, 18), (2, 3), (1, 1), (96, 40), (100, 80)):
        for omega in (1.0, 1.3):
            wl = scalar_case(*shape, BC_SETS[bcname], omega, 0, seed=5)
            s = Solver.from_workload(wl, precision="f32")
            s.set_state(torch.from_numpy(wl.prim).cuda())
            for n in (1, 2, 7, 70):
                s.step(n)
                out.append(s.get_distributions().cpu().numpy().ravel())
            s.close()
np.save(sys.argv[2], np.concatenate(out))
"""


def test_f32_two_step_kernel_equals_single_steps(tmp_path):
    """FP32 scalar D2Q4 advances two steps per launch (step2ds_fused2_kernel: the window's step n+1
    in shared memory, then the tile's step n+2, with the single-step kernel's pull and collision);
    the state must equal one step per launch (LBRS_F32S_FUSE=0) bit for bit on every side set,
    ragged and one-cell grids, odd and even step counts and graph replay, at every tile height the
    kernel takes (32 rows by default, 16 and 24 through LBRS_F32S_TILE_Y).  Interior tiles, which load
    on direct offsets, occur on the 96 x 40 grid at 16 rows and on the 100 x 80 grid at every height."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "scalar_fuse.py"
    script.write_text(_FUSE_SCRIPT)
    res = {}
    runs = (("fused", {}), ("fused16", {"LBRS_F32S_TILE_Y": "16"}), ("fused24", {"LBRS_F32S_TILE_Y": "24"}),
            ("single", {"LBRS_F32S_FUSE": "0"}))
    for name, env_add in runs:
        out = tmp_path / f"{name}.npy"
        subprocess.run([sys.executable, str(script), root, str(out)], check=True, env=dict(os.environ, **env_add),
                       timeout=600)
        res[name] = np.load(out)
    assert np.all(np.isfinite(res["single"]))
    for name in ("fused", "fused16", "fused24"):
        assert np.array_equal(res[name], res["single"]), (name, np.max(np.abs(res[name] - res["single"])))
