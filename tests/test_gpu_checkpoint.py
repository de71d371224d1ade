"""Checkpoint blobs through the C ABI: resuming is bit-identical to an uninterrupted run (device
and host blobs, the FP32, FP64 and FP16 forms, the two-steps-per-launch path, the step counter);
a blob of another configuration or a foreign buffer is refused."""
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()


def solver(wl, precision, **kw):
    from paper_1504_07034_gb300.solver import Solver
    return Solver.from_workload(wl, precision=precision, **kw)


@pytest.mark.parametrize("precision", ["f64", "f32", "f16neq"])
@pytest.mark.parametrize("device", [True, False])
def test_resume_is_bitwise(precision, device):
    wl = W.oblique_shock_reflection(nx=128, ny=32, steps=0, omega=1.3)
    a = solver(wl, precision)
    a.set_state(torch.from_numpy(wl.prim).cuda())
    a.step(31)
    blob = a.checkpoint(device=device)
    a.step(77)
    want = a.get_distributions().clone()
    b = solver(wl, precision)
    b.restore(blob)
    assert b.step_count == 31
    b.step(77)
    assert torch.equal(b.get_distributions(), want)
    assert b.step_count == a.step_count == 108
    a.close()
    b.close()


def test_foreign_or_mismatched_blobs_are_refused():
    from paper_1504_07034_gb300 import abi
    wl = W.quadrant_riemann(1, 48, steps=0)
    a = solver(wl, "f32")
    a.set_state(torch.from_numpy(wl.prim).cuda())
    a.step(5)
    blob = a.checkpoint()
    other = solver(wl, "f32", omega=1.2)
    with pytest.raises(abi.LbrsError) as e:
        other.restore(blob)
    assert e.value.status == abi.LBRS_EINVAL
    other.close()
    bad = blob.clone()
    bad[0] = ord("X")
    with pytest.raises(abi.LbrsError):
        a.restore(bad)
    a.close()
