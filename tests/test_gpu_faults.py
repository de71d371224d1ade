"""Faults injected on the host, detected by the library (nothing faults, traps or hangs the GPU).

* Non-physical input fields -- a cell with negative pressure, one with negative density, one
  holding a NaN -- are counted by the diagnostics at step 0 (LBRS_ENONPHYS, exactly those cells),
  in every storage form that has diagnostics.
* With periodic checks on, a run started from such a field reports LBRS_ENONPHYS at the first
  checked step through lbrs_sync, and a healthy state set afterwards clears the record.
* A bounded device wait that runs out (on an mbarrier that nothing completes, the self-test
  launch) raises the workspace flag; lbrs_sync reports LBRS_ETIMEOUT and a new state clears it.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

BAD = [(5, 7), (20, 3), (33, 30)]          # (i, j): p < 0, rho < 0, NaN


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()


def poisoned(n=48):
    wl = W.quadrant_riemann(3, n, steps=0)
    prim = wl.prim.copy()
    (i0, j0), (i1, j1), (i2, j2) = BAD
    prim[3, j0, i0] = -0.2
    prim[0, j1, i1] = -0.5
    prim[1, j2, i2] = np.nan
    return wl, prim


@pytest.mark.parametrize("precision", ["f64", "f32", "f16neq", "f32u"])
def test_nonphysical_input_counted_at_step_zero(precision):
    from paper_1504_07034_gb300.solver import Solver
    wl, prim = poisoned()
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(prim).cuda())
    d = s.diagnostics()
    assert d["status"] == "LBRS_ENONPHYS"
    assert d["n_nonphysical"] == len(BAD)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    d = s.diagnostics()
    assert d["status"] == "LBRS_OK" and d["n_nonphysical"] == 0
    s.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_nonphysical_input_reported_by_periodic_checks(precision):
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl, prim = poisoned()
    s = Solver.from_workload(wl, precision=precision, diag_every=2)
    s.set_state(torch.from_numpy(prim).cuda())
    s.step(7)
    with pytest.raises(abi.LbrsError) as e:
        s.sync()
    assert e.value.status == abi.LBRS_ENONPHYS
    assert s.first_bad_step() == 2
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(7)
    s.sync()
    assert s.first_bad_step() == -1
    s.close()


def test_bounded_wait_runs_out_and_is_reported():
    """A bounded device wait on an mbarrier that nothing completes gives up and raises the
    workspace flag (the self-test launch); lbrs_sync reports LBRS_ETIMEOUT, the context stays
    usable, and a new state clears the flag."""
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl = W.quadrant_riemann(0, 64, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(4)
    s.sync()
    f_before = s.get_distributions().clone()
    abi.check(s.lib.lbrs_selftest_wait_timeout(s.ctx))
    with pytest.raises(abi.LbrsError) as e:
        s.sync()
    assert e.value.status == abi.LBRS_ETIMEOUT
    assert torch.equal(s.get_distributions(), f_before)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(4)
    s.sync()
    assert torch.equal(s.get_distributions(), f_before)
    s.close()
