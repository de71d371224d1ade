"""The FP16 non-equilibrium storage form (LBRS_F16NEQ) against the FP64 oracle.

Per cell it keeps U in FP32 and the post-collision non-equilibrium parts of
three populations per field in FP16.  At omega = 1 those parts vanish (the
post-collision state is f^eq(U)), so the form reduces to FP32 arithmetic on U;
at omega != 1 the FP16 rounding of the non-equilibrium parts enters.  The
density L1 error against the FP64 oracle is stated and bounded.
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
    d = s.diagnostics()
    s.close()
    return U, d


def oracle_U(wl):
    o = oracle.Oracle.from_workload(wl)
    fs, _ = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps)
    return o.moments(fs)


def small(bc, omega, nx=160, ny=96, steps=120):
    from test_gpu_parity import small_case
    return small_case(nx, ny, bc, omega, steps=steps)


@pytest.mark.parametrize("bc", ["transmissive", "periodic", "dirichlet_wall", "walls_periodic_x", "mixed"])
@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_f16neq_close_to_oracle(bc, omega):
    wl = small(bc, omega)
    ref = oracle_U(wl)
    U16, d = run(wl, "f16neq")
    U32, _ = run(wl, "f32")
    l1_16 = float(np.mean(np.abs(U16[0] - ref[0])))
    l1_32 = float(np.mean(np.abs(U32[0] - ref[0])))
    print(f"{bc} omega={omega}: density L1 vs FP64 oracle: f16neq {l1_16:.2e}, f32 {l1_32:.2e}")
    assert d["status"] == "LBRS_OK"
    assert l1_16 <= (1e-5 if omega == 1.0 else 2e-4)


def test_f16neq_at_omega1_matches_f32_closely():
    wl = small("transmissive", 1.0)
    U16, _ = run(wl, "f16neq")
    U32, _ = run(wl, "f32")
    assert np.max(np.abs(U16 - U32)) <= 1e-5 * np.max(np.abs(U32))


def test_f16neq_checkpoint_roundtrip_and_diagnostics():
    from paper_1504_07034_gb300.solver import Solver
    wl = small("dirichlet_wall", 1.5, steps=0)
    a = Solver.from_workload(wl, precision="f16neq")
    a.set_state(torch.from_numpy(wl.prim).cuda())
    a.step(30)
    raw = a.raw_state().clone()
    a.step(25)
    end = a.moments()
    b = Solver.from_workload(wl, precision="f16neq")
    b.set_raw_state(raw, step=30)
    b.step(25)
    assert torch.equal(b.moments(), end)
    o = oracle.Oracle.from_workload(wl)
    d = a.diagnostics()
    assert d["totals"][0] == pytest.approx(float(end[0].sum()) * wl.dx * wl.dx, rel=1e-12)
    a.close()
    b.close()


def test_f16neq_rejected_where_undefined():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    with pytest.raises(abi.LbrsError):
        Solver("d1q2", 32, lam=3.0, dx=1 / 32, bc=[("transmissive", None)] * 2, precision="f16neq")
    wl, _ = W.adjoint_pulses(n=16, steps=0)
    s = Solver.from_workload(wl, precision="f16neq")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    with pytest.raises(abi.LbrsError):
        s.forward_checkpointed(4, 2)
    s.close()


@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_full_size_oblique_shock_f16neq(omega):
    """4096 x 1024 oblique shock reflection, 150 steps (the oracle's share at full size)."""
    wl = W.oblique_shock_reflection(steps=150, omega=omega)
    ref = oracle_U(wl)
    U16, d = run(wl, "f16neq")
    l1 = float(np.mean(np.abs(U16[0] - ref[0])))
    print(f"oblique 4096x1024 x150 omega={omega}: f16neq density L1 vs FP64 oracle {l1:.2e}")
    assert d["status"] == "LBRS_OK"
    assert l1 <= 1e-4
