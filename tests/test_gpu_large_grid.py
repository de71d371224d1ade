"""A grid past the 32-bit element range: 16384 x 8256 cells, so that the 16 distribution planes hold
2.16e9 values per buffer and every plane offset beyond the first needs 64-bit arithmetic.

The state is a patchwork of three constant states chosen by integer cell coordinates (so both sides
build it exactly), under transmissive, Dirichlet and wall sides.  After 5 steps (two two-step
launches and one single step in FP32; single steps in FP64) the distributions of sampled cells --
among them the grid's corners and the last rows, whose element offsets are the largest -- are
compared with the oracle run on a crop around each sample: after n steps a cell depends only on
cells within n cells of it (each move is one cell in x and in y), so a crop with that margin, the
domain's own sides where it touches them, gives the cell's exact value.  FP64 to 1e-12 of the
largest distribution, FP32 to 2e-6.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

NX, NY, STEPS = 16384, 8256, 5
LAM, GAMMA, OMEGA = 4.0, 1.4, 1.3
STATES = np.array([[1.0, 0.3, -0.2, 1.0], [0.5, -0.4, 0.1, 0.6], [0.8, 0.0, 0.5, 1.4]])
BC = [("dirichlet", (1.1, 0.4, 0.0, 1.2)), ("transmissive", None), ("wall", None), ("transmissive", None)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()
    oracle.build()


def pattern(i, j):
    """State index of cell (i, j): bands of 37 columns and 53 rows."""
    return (i // 37 + j // 53) % 3


def prim_of(i, j):
    """Primitive fields of the cells (i, j) (numpy index arrays); v = 0 on the wall row."""
    p = STATES[pattern(i, j)].transpose(np.roll(np.arange(np.ndim(i) + 1), 1)).copy()
    p[2] = np.where(j == 0, 0.0, p[2])
    return p


def device_prim():
    j = torch.arange(NY, device="cuda", dtype=torch.int64)[:, None]
    i = torch.arange(NX, device="cuda", dtype=torch.int64)[None, :]
    idx = (torch.div(i, 37, rounding_mode="floor") + torch.div(j, 53, rounding_mode="floor")) % 3
    st = torch.from_numpy(STATES).cuda()
    prim = st[idx].permute(2, 0, 1).contiguous()
    prim[2, 0, :] = 0.0
    return prim


SAMPLES = [(0, 0), (NX - 1, 0), (0, NY - 1), (NX - 1, NY - 1), (NX - 2, NY - 3), (3, NY - 1), (NX - 1, 4),
           (8191, 4127), (12345, 8000), (16000, 8255), (37 * 300, 53 * 120), (37 * 300 - 1, 53 * 120 - 1),
           (5, 2), (16383, 8254), (9000, 1)]


def oracle_cell(i, j):
    """Distributions [16] of cell (i, j) after STEPS steps, from the oracle on a crop."""
    m = STEPS + 1
    i0, i1 = max(0, i - m), min(NX, i + m + 1)
    j0, j1 = max(0, j - m), min(NY, j + m + 1)
    T = ("transmissive", None)
    bc = [BC[0] if i0 == 0 else T, BC[1] if i1 == NX else T, BC[2] if j0 == 0 else T, BC[3] if j1 == NY else T]
    jj, ii = np.meshgrid(np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
    o = oracle.Oracle(oracle.D2Q4, i1 - i0, j1 - j0, lam=LAM, omega=OMEGA, gamma=GAMMA, bc=bc, dx=1.0 / NX)
    fs, _ = o.run(o.init(o.prim_to_cons(prim_of(ii, jj))), STEPS)
    return fs[:, :, j - j0, i - i0].reshape(16)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_grid_past_32_bit_offsets(precision):
    from paper_1504_07034_gb300.solver import Solver
    assert 16 * NX * NY > 2 ** 31
    s = Solver("d2q4", NX, NY, lam=LAM, dx=1.0 / NX, bc=BC, gamma=GAMMA, omega=OMEGA, precision=precision)
    s.set_state(device_prim())
    s.step(STEPS)
    s.sync()
    f = s.get_distributions()
    idx_j = torch.tensor([j for _, j in SAMPLES], device="cuda")
    idx_i = torch.tensor([i for i, _ in SAMPLES], device="cuda")
    got = f[:, :, idx_j, idx_i].double().cpu().numpy().reshape(16, -1).T
    s.close()
    del f
    torch.cuda.empty_cache()
    want = np.array([oracle_cell(i, j) for i, j in SAMPLES])
    scale = np.abs(want).max()
    tol = 1e-12 if precision == "f64" else 2e-6
    err = np.abs(got - want).max(axis=1) / scale
    assert np.all(err <= tol), dict(zip(SAMPLES, err))
