"""GPU parity of the adaptive lattice speed (D2Q4) through the C ABI.

Bars: FP64 against the oracle's adaptive run: the same number of steps, the same time reached
and final lambda (to 1e-12; both evaluate the same expressions in the same order), the
distributions to 1e-12 normwise; FP32 against the oracle to 2e-5 normwise on the moments.
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


def normwise(a, b, axis):
    """Largest |a - b| relative to the largest |b|, taken per conserved field (axis: the field
    axis of the arrays; a field that is zero throughout is scaled by the largest of all)."""
    a, b = np.moveaxis(np.asarray(a), axis, 0), np.moveaxis(np.asarray(b), axis, 0)
    glob = float(np.max(np.abs(b)))
    return max(float(np.max(np.abs(a[k] - b[k]))) / (float(np.max(np.abs(b[k]))) or glob) for k in range(b.shape[0]))


CASES = {
    "quadrants": (lambda: W.quadrant_riemann(2, 64, steps=0), 1.05, 0.3),
    "oblique": (lambda: W.oblique_shock_reflection(nx=96, ny=24, steps=0), 1.1, 0.3),
    "periodic": (lambda: W.adjoint_pulses(seed=1, n=48, steps=0, width=0.1, pulses=3)[0], 1.2, 0.0),
}


def oracle_adaptive(wl, safety, t_final, nsteps):
    o = oracle.Oracle.from_workload(wl)
    fs, lam, t, lam_next = o.run_adaptive(o.init(o.prim_to_cons(wl.prim)), nsteps, wl.dx, safety, t_final)
    return fs, o.moments(fs), len(lam), t, lam_next


def gpu_adaptive(wl, precision, safety, t_final, nsteps):
    from paper_1504_07034_gb300.solver import Solver
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    if t_final > 0:
        st = s.run_to_time(t_final, safety, chunk=40)   # a 32-step graph and 8 single steps per chunk
    else:
        s.step_adaptive(nsteps, safety)
        st = s.adaptive_state()
    fs = s.get_distributions().double().cpu().numpy()
    U = s.moments(torch.float64).cpu().numpy()
    s.close()
    return fs, U, st


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_f64_adaptive_matches_oracle(case, omega):
    make, safety, t_final = CASES[case]
    wl = make()
    wl.omega = omega
    fr, Ur, n, t, lam_next = oracle_adaptive(wl, safety, t_final, 70 if t_final == 0 else 10 ** 6)
    fs, U, st = gpu_adaptive(wl, "f64", safety, t_final, 70)
    assert st["steps"] == n
    assert st["t"] == pytest.approx(t, rel=1e-12)
    assert st["lambda"] == pytest.approx(lam_next, rel=1e-12)
    assert st["done"] == (t_final > 0)
    if t_final > 0:
        assert st["t"] == t_final
    assert normwise(fs, fr, 1) <= 1e-12
    assert normwise(U, Ur, 0) <= 1e-12


@pytest.mark.parametrize("case", ["quadrants", "oblique"])
def test_f32_adaptive_close_to_oracle(case):
    make, safety, t_final = CASES[case]
    wl = make()
    _, Ur, n, t, _ = oracle_adaptive(wl, safety, t_final, 10 ** 6)
    _, U, st = gpu_adaptive(wl, "f32", safety, t_final, 0)
    assert st["t"] == t_final
    assert abs(st["steps"] - n) <= 1
    if st["steps"] == n:
        assert normwise(U, Ur, 0) <= 2e-5


def test_after_the_end_steps_keep_the_state_and_a_new_state_resets():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    make, safety, t_final = CASES["oblique"]
    wl = make()
    s = Solver.from_workload(wl, precision="f64")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    st = s.run_to_time(t_final, safety, chunk=8)
    f_end = s.get_distributions().clone()
    s.step_adaptive(5, safety, t_final)
    assert torch.equal(s.get_distributions(), f_end)
    assert s.adaptive_state() == st
    # fixed-lambda steps are refused while the distributions carry an adaptive lambda
    with pytest.raises(abi.LbrsError) as e:
        s.step(1)
    assert e.value.status == abi.LBRS_ESTATE
    # a new state restores the configured lambda and its ghosts: equal to a fresh solver
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(40)
    fresh = Solver.from_workload(wl, precision="f64")
    fresh.set_state(torch.from_numpy(wl.prim).cuda())
    fresh.step(40)
    assert torch.equal(s.get_distributions(), fresh.get_distributions())
    s.close()
    fresh.close()


def test_adaptive_rejections():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl = W.quadrant_riemann(2, 32, steps=0)
    s = Solver.from_workload(wl, precision="f32")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    with pytest.raises(abi.LbrsError):
        s.step_adaptive(1, safety=0.9)
    with pytest.raises(abi.LbrsError):
        s.step_adaptive(1, safety=1.0, t_final=0.5 * wl.dx / wl.lam)   # the first step passes t_final
    m = np.zeros((32, 32), np.uint8)
    m[10:14, 10:14] = 1
    s.set_obstacles(m)
    with pytest.raises(abi.LbrsError):
        s.step_adaptive(1)
    s.close()
    s = Solver.from_workload(W.burgers_2d(1, 32), precision="f64")
    s.set_state(torch.from_numpy(W.burgers_2d(1, 32).prim).cuda())
    with pytest.raises(abi.LbrsError):
        s.step_adaptive(1)
    s.close()
