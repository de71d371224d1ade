"""lbrs_diagnostics_noalloc: diagnostics for callers that cannot allocate device memory.

Loops that must not stall on cudaMalloc's implicit synchronisation and
processes whose device memory is held by another allocator cannot hand the
library a workspace.  The allocation-free entry point keeps its reduction
scratch in a static device array instead.  These tests call it through the C
ABI and check it against the workspace-based lbrs_diagnostics on the same
distributions, for each accepted lattice, twice in a row (the scratch is
shared and keeps the previous call's contents).

This file is named so that pytest collects it last.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12   # the totals are summed in a different (but fixed) block order


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()


def _solver(lattice, precision):
    from paper_1504_07034_gb300.solver import Solver
    if lattice == "d2q4":
        wl = W.quadrant_riemann(2, 320, steps=60)
        wl.prim = np.ascontiguousarray(wl.prim[:, :200, :])      # ragged 320 x 200 grid
        wl.ny = 200
        s = Solver.from_workload(wl, precision=precision)
    else:
        wl = W.sod(5000, lattice=lattice)
        s = Solver.from_workload(wl, precision=precision, lattice=lattice)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(60 if lattice == "d2q4" else wl.steps)
    return s


def _noalloc(s, fs):
    from paper_1504_07034_gb300 import abi
    d = abi.lbrs_diag()
    st = abi.load().lbrs_diagnostics_noalloc(ctypes.byref(s.cfg), ctypes.c_void_p(fs.data_ptr()), ctypes.byref(d))
    return st, d


def _same(ref, d, K):
    assert np.allclose([d.totals[k] for k in range(K)], ref["totals"], rtol=RTOL, atol=0.0)
    assert d.min_rho == ref["min_rho"]
    assert d.min_p == ref["min_p"]
    assert d.max_lambda_local == ref["max_lambda_local"]
    assert d.n_nonphysical == ref["n_nonphysical"] and d.n_subchar == ref["n_subchar"]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("lattice", ["d2q4", "d1q2", "d1q3"])
def test_noalloc_matches_workspace_diagnostics_twice(lattice, precision):
    from paper_1504_07034_gb300 import abi
    s = _solver(lattice, precision)
    ref = s.diagnostics()
    fs = s.get_distributions()
    gc.collect()                      # objects left by earlier tests must not be freed mid-check
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    first = None
    for _ in range(2):
        st, d = _noalloc(s, fs)
        assert abi.status_name(st) == ref["status"], abi.load().lbrs_last_error(None)
        _same(ref, d, s.K)
        if first is None:
            first = [d.totals[k] for k in range(4)]
        else:
            assert [d.totals[k] for k in range(4)] == first      # bitwise repeatable
    assert torch.cuda.memory_allocated() <= before      # the entry point allocated nothing through torch
    s.close()


def test_noalloc_second_call_on_smaller_grid_is_not_stale():
    """A call on a grid needing fewer partial records must not see the previous call's records."""
    from paper_1504_07034_gb300 import abi
    big = _solver("d2q4", "f32")
    small = _solver("d1q2", "f32")
    ref_big, ref_small = big.diagnostics(), small.diagnostics()
    st, d = _noalloc(big, big.get_distributions())
    assert abi.status_name(st) == ref_big["status"]
    _same(ref_big, d, big.K)
    st, d = _noalloc(small, small.get_distributions())
    assert abi.status_name(st) == ref_small["status"]
    _same(ref_small, d, small.K)
    big.close()
    small.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import make_config
    cfg = make_config("d2q4", 8192, 8192, gamma=1.4, lam=3.0, omega=1.0, dx=1 / 8192,
                      bc=[("transmissive", None)] * 4, precision="f32", stream_handle=0)
    dummy = torch.empty(16, device="cuda")
    d = abi.lbrs_diag()
    st = abi.load().lbrs_diagnostics_noalloc(ctypes.byref(cfg), ctypes.c_void_p(dummy.data_ptr()), ctypes.byref(d))
    assert st == abi.LBRS_EINVAL
    msg = abi.load().lbrs_last_error(None).decode()
    assert "33554432" in msg and "no-allocation" in msg
