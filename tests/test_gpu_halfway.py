"""The halfway free-slip wall on the GPU (LBRS_BC_WALL_HALFWAY).

Parity with the oracle (FP64 <= 1e-12 per field, FP32 density L1) runs with the other
boundary sets in test_gpu_parity.py, the two-step kernels' bit-identity to single steps
in its kernel-variant test, and the y-slab split in test_gpu_slabs.py.  Here: the GPU
path's own mirror-doubled check (a walled grid is the lower half of the periodic grid of
twice its height that holds its mirror image), and the configurations that are refused.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()


def _fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid((np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx, indexing="ij")
    w = np.empty((4, ny, nx))
    w[0] = 1.0 + 0.2 * np.sin(2 * np.pi * (x + rng.uniform())) * np.cos(np.pi * (y + rng.uniform()))
    w[1] = 0.3 + 0.2 * np.cos(2 * np.pi * (x + y + rng.uniform()))
    w[2] = 0.2 * np.sin(2 * np.pi * (2 * x + rng.uniform())) * np.sin(np.pi * y)
    w[3] = 1.0 + 0.3 * np.cos(2 * np.pi * (x - y + rng.uniform())) ** 2
    return w


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 1e-5)])
@pytest.mark.parametrize("nx", [64, 66])               # tensor-copy and direct-load two-step kernels
def test_walled_grid_is_half_of_the_mirror_doubled_grid(precision, tol, nx):
    from paper_1504_07034_gb300.solver import Solver
    ny, steps = 40, 60
    w = _fields(nx, ny, 11)
    wd = np.concatenate([w, w[:, ::-1, :]], axis=1)
    wd[2, ny:] *= -1.0
    xs = [("transmissive", None), ("transmissive", None)]
    a = Solver("d2q4", nx, ny, lam=4.0, dx=1.0 / ny, bc=xs + [("wall_halfway", None)] * 2, omega=1.3,
               precision=precision)
    b = Solver("d2q4", nx, 2 * ny, lam=4.0, dx=1.0 / ny, bc=xs + [("periodic", None)] * 2, omega=1.3,
               precision=precision)
    for s, f in ((a, w), (b, wd)):
        s.set_state(torch.from_numpy(np.ascontiguousarray(f)).cuda())
        s.step(steps)
    Ua = a.moments(torch.float64).cpu().numpy()
    Ub = b.moments(torch.float64).cpu().numpy()
    for k in range(4):
        scale = np.max(np.abs(Ub[k]))
        assert np.max(np.abs(Ua[k] - Ub[k, :ny])) <= tol * scale, k
    a.close()
    b.close()


def test_halfway_walls_refused_where_not_defined():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    bc = [("periodic", None)] * 2 + [("wall_halfway", None)] * 2
    for precision in ("f16neq", "f32u"):
        with pytest.raises(abi.LbrsError):
            Solver("d2q4", 32, 16, lam=4.0, dx=1 / 32, bc=bc, precision=precision)
    with pytest.raises(abi.LbrsError):
        Solver("d2q4", 32, 16, lam=4.0, dx=1 / 32, bc=[("wall_halfway", None)] * 4, precision="f32")
    with pytest.raises(abi.LbrsError):
        Solver("d1q2", 32, lam=4.0, dx=1 / 32, bc=[("wall_halfway", None)] * 2, precision="f32")
    s = Solver("d2q4", 32, 16, lam=4.0, dx=1 / 32, bc=bc, precision="f32")
    with pytest.raises(abi.LbrsError):
        s.set_obstacles(torch.zeros((16, 32), dtype=torch.uint8))
    s.close()
