"""The boundary balance of a step (lbrs_boundary_flux) against the step itself.

Streaming moves every population to x + c_q; the ones whose destination lies beyond a
non-periodic side leave (outflow), and the cells whose pull source lies beyond one receive
what the side condition gives them (inflow); the collision keeps the moments.  So the FP64
totals after one step must equal the totals before plus inflow minus outflow, for every
side kind and corner combination, in both storage precisions.  The outflow is also summed
here on the host from the distributions, independently of the library.
"""
import numpy as np
import pytest
import torch

import workloads as W
from test_gpu_parity import BC_SETS, small_case

pytestmark = pytest.mark.gpu

SX = (-1, 1, 1, -1)
SY = (-1, -1, 1, 1)


def host_outflow(f, bc, dx):
    """Sum over the side cells of the populations whose destination x + c_q leaves the grid."""
    Q, K, ny, nx = f.shape
    px, py = bc[0][0] == "periodic", bc[2][0] == "periodic"
    out = np.zeros(K)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for q in range(4):
        di, dj = ii + SX[q], jj + SY[q]
        leaves = np.zeros((ny, nx), dtype=bool)
        if not px:
            leaves |= (di < 0) | (di >= nx)
        if not py:
            leaves |= (dj < 0) | (dj >= ny)
        for k in range(K):
            out[k] += float(np.sum(f[q, k][leaves], dtype=np.float64))
    return out * dx * dx


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
@pytest.mark.parametrize("shape", [(64, 40), (37, 29), (1, 9), (33, 1)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_step_changes_totals_by_the_boundary_balance(bcname, shape, precision):
    from paper_1504_07034_gb300.solver import Solver
    nx, ny = shape
    bc = BC_SETS[bcname]
    if bc[0][0] == "periodic" and nx % 2:
        nx += 1
    if bc[2][0] == "periodic" and ny % 2:
        ny += 1
    if any(kind == "wall" for kind, _ in bc[2:]):
        ny = max(ny, 2)
    wl = small_case(nx, ny, bcname, 1.0, steps=10)
    s = Solver("d2q4", nx, ny, lam=wl.lam, dx=wl.dx, bc=bc, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    for n in (0, 7, 1, 3):
        s.step(n)
        t0 = np.array(s.diagnostics()["totals"])
        flux = s.boundary_flux()
        again = s.boundary_flux()
        assert again == flux                                    # fixed order: bitwise repeatable
        fin, fout = np.array(flux["inflow"]), np.array(flux["outflow"])
        f = s.get_distributions().double().cpu().numpy()
        ref_out = host_outflow(f, bc, wl.dx)
        # one scale for all fields: a field whose total nearly cancels (x-momentum) keeps the
        # rounding of the magnitudes summed into it
        scale = np.max(np.abs(t0)) + np.max(np.abs(fin)) + np.max(np.abs(fout))
        tol = 1e-13 if precision == "f64" else 1e-6
        assert np.all(np.abs(fout - ref_out) <= tol * scale), (fout, ref_out)
        s.step(1)
        t1 = np.array(s.diagnostics()["totals"])
        assert np.all(np.abs((t1 - t0) - (fin - fout)) <= (1e-12 if precision == "f64" else 1e-6) * scale), \
            (t1 - t0, fin - fout)
        if bcname == "periodic":
            assert not np.any(fin) and not np.any(fout)
    s.close()


def test_balance_over_a_run_of_the_oblique_shock():
    """Over 40 FP64 steps of a coarse oblique shock reflection (Dirichlet inflow and top, transmissive
    outflow, wall below), the sum of the per-step balances accounts for the change of the totals."""
    from paper_1504_07034_gb300.solver import Solver
    wl = W.oblique_shock_reflection(nx=256, ny=64, steps=40)
    s = Solver.from_workload(wl, precision="f64")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    t_start = np.array(s.diagnostics()["totals"])
    net = np.zeros(4)
    for _ in range(wl.steps):
        fl = s.boundary_flux()
        net += np.array(fl["inflow"]) - np.array(fl["outflow"])
        s.step(1)
    t_end = np.array(s.diagnostics()["totals"])
    assert np.any(np.abs(net) > 1e-3 * np.abs(t_start))           # the sides do exchange
    # y-momentum starts at exactly zero: one scale, that of the largest total, for all fields
    assert np.all(np.abs((t_end - t_start) - net) <= 1e-12 * np.max(np.abs(t_start)))
    s.close()


def test_balance_rejects_forms_it_does_not_cover():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl = small_case(32, 16, "transmissive", 1.0, steps=1)
    for precision in ("f32u", "f16neq"):
        s = Solver("d2q4", 32, 16, lam=wl.lam, dx=wl.dx, bc=wl.bc, precision=precision)
        s.set_state(torch.from_numpy(wl.prim).cuda())
        with pytest.raises(abi.LbrsError) as e:
            s.boundary_flux()
        assert e.value.status == abi.LBRS_EINVAL
        s.close()
    s = Solver("d2q4", 32, 16, lam=wl.lam, dx=wl.dx, bc=wl.bc, precision="f64")
    with pytest.raises(abi.LbrsError) as e:                         # no state yet
        s.boundary_flux()
    assert e.value.status == abi.LBRS_ESTATE
    s.close()


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
@pytest.mark.parametrize("shape", [(64, 40), (37, 29)])
def test_f64_balance_equals_the_oracles(bcname, shape):
    """The FP64 library's inflow and outflow against the oracle's (orc_boundary_flux) after five steps of
    the same state: the same populations summed in another order."""
    import oracle
    from paper_1504_07034_gb300.solver import Solver
    nx, ny = shape
    bc = BC_SETS[bcname]
    if bc[0][0] == "periodic" and nx % 2:
        nx += 1
    if bc[2][0] == "periodic" and ny % 2:
        ny += 1
    wl = small_case(nx, ny, bcname, 1.3, steps=5)
    o = oracle.Oracle.from_workload(wl)
    fs, _ = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps)
    fin_o, fout_o = o.boundary_flux(fs, wl.dx * wl.dx)
    s = Solver.from_workload(wl, precision="f64")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(wl.steps)
    flux = s.boundary_flux()
    s.close()
    scale = np.max(np.abs(fin_o)) + np.max(np.abs(fout_o))
    assert np.all(np.abs(np.array(flux["inflow"]) - fin_o) <= 1e-12 * scale), (flux["inflow"], fin_o)
    assert np.all(np.abs(np.array(flux["outflow"]) - fout_o) <= 1e-12 * scale), (flux["outflow"], fout_o)
