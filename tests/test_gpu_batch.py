"""GPU parity of the batched D1Q2 tubes (temporal blocking) through the C ABI.

Every tube of a batch must evolve exactly as a lone tube: the FP64 batched path
against the FP64 oracle run tube by tube to 1e-12 (normwise per field), for
several launch shapes (tile, block, halo), ragged lengths (1 cell up to
several tiles), zero-step tubes, periodic ends and repeated runs.  FP32
against the oracle: density L1 per tube.  At the full 4096-tube size a
sample of tubes (the longest among them) is checked against the oracle.
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


def small_batch(seed, count=23, n_min=1, n_max=700):
    tb = W.batched_tubes(seed=seed, count=count, n_min=max(n_min, 1), n_max=n_max, t_final=0.15)
    rng = np.random.default_rng(seed)
    steps = rng.integers(0, 300, size=count)
    steps[rng.integers(0, count)] = 0
    return tb, steps


def oracle_tube(tb, b, steps, prim_all, offsets, boundary="transmissive"):
    n = int(tb.lengths[b])
    o = oracle.Oracle(oracle.D1Q2, n, lam=float(tb.lam[b]), omega=tb.omega, gamma=tb.gamma,
                      bc=[(boundary, None)] * 2)
    prim = prim_all[:, offsets[b]:offsets[b] + n]
    fs, _ = o.run(o.init(o.prim_to_cons(prim)), int(steps))
    return o.moments(fs)


def run_batch(tb, steps, precision, tuning=None, boundary="transmissive", prim=None, repeat=1):
    from paper_1504_07034_gb300.solver import BatchSolver
    s = BatchSolver(tb.lengths, tb.lam, gamma=tb.gamma, omega=tb.omega, boundary=boundary, precision=precision)
    if tuning:
        s.tuning = tuning
    s.set_state(torch.from_numpy(tb.prim() if prim is None else prim).cuda())
    for _ in range(repeat):
        s.run(steps)
    U = s.moments().cpu().numpy()
    s.close()
    return U


def check_f64(U, tb, steps, prim, boundary="transmissive"):
    off = np.concatenate([[0], np.cumsum(tb.lengths)[:-1]])
    for b in range(len(tb.lengths)):
        ref = oracle_tube(tb, b, steps[b], prim, off, boundary)
        got = U[:, off[b]:off[b] + tb.lengths[b]]
        err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref))
        assert np.all(err <= 1e-12), (b, tb.lengths[b], steps[b], err)


@pytest.mark.parametrize("tuning", [None, (128, 1, 8), (256, 4, 32), (512, 2, 64), (128, 8, 16)])
def test_f64_batch_matches_oracle_per_tube(tuning):
    tb, steps = small_batch(1)
    U = run_batch(tb, steps, "f64", tuning)
    check_f64(U, tb, steps, tb.prim())


def test_f64_batch_periodic_tubes():
    tb, steps = small_batch(2, count=12, n_min=1, n_max=300)
    rng = np.random.default_rng(2)
    prim = tb.prim()
    prim[0] *= 1 + 0.2 * rng.uniform(-1, 1, prim.shape[1])            # break the symmetry of the tubes
    tb.lam = tb.lam * 1.5
    U = run_batch(tb, steps, "f64", (128, 2, 16), boundary="periodic", prim=prim)
    check_f64(U, tb, steps, prim, boundary="periodic")


def test_repeated_runs_equal_one_long_run():
    tb, steps = small_batch(3, count=9)
    U2 = run_batch(tb, steps, "f64", (256, 2, 16), repeat=2)
    U1 = run_batch(tb, 2 * steps, "f64", (256, 2, 16))
    assert np.array_equal(U1, U2)


def test_f32_batch_close_to_oracle_and_tunings_agree():
    tb, steps = small_batch(4)
    prim = tb.prim()
    Ua = run_batch(tb, steps, "f32", (256, 2, 16))
    Ub = run_batch(tb, steps, "f32", (128, 8, 64))
    assert np.max(np.abs(Ua - Ub)) <= 1e-6 * np.max(np.abs(Ua))
    off = np.concatenate([[0], np.cumsum(tb.lengths)[:-1]])
    for b in range(len(tb.lengths)):
        ref = oracle_tube(tb, b, steps[b], prim, off)
        got = Ua[:, off[b]:off[b] + tb.lengths[b]]
        assert np.mean(np.abs(got[0] - ref[0])) <= 1e-6


def test_autotune_keeps_state_and_returns_valid_tuning():
    from paper_1504_07034_gb300.solver import BatchSolver
    tb, steps = small_batch(5, count=40, n_min=50, n_max=3000)
    s = BatchSolver(tb.lengths, tb.lam, gamma=tb.gamma, omega=tb.omega, precision="f32")
    s.set_state(torch.from_numpy(tb.prim()).cuda())
    before = s.get_distributions().clone()
    tuning, ns = s.autotune(np.maximum(steps, 1))
    assert torch.equal(before, s.get_distributions())
    block, cpt, halo = tuning
    assert block in (128, 256, 512) and block * cpt - 2 * halo >= 32 and ns > 0
    s.run(steps)
    U = s.moments().cpu().numpy()
    s.close()
    Uref = run_batch(tb, steps, "f32", (256, 2, 16))
    assert np.max(np.abs(U - Uref)) <= 1e-6 * np.max(np.abs(Uref))


def test_batch_rejects_bad_arguments():
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import BatchSolver
    with pytest.raises(abi.LbrsError):
        BatchSolver([10, 0], [1.0, 1.0])
    s = BatchSolver([10, 20], [2.0, 2.0])
    with pytest.raises(abi.LbrsError) as e:
        s.run([1, 1])
    assert e.value.status == abi.LBRS_ESTATE
    with pytest.raises(abi.LbrsError):
        s.tuning = (256, 1, 200)
    s.close()


def test_full_size_batch_sampled_against_oracle():
    """4096 tubes (N log-uniform in [200, 20000]) to t = 0.15 in FP32; sampled tubes vs the FP64 oracle."""
    tb = W.batched_tubes(seed=0, count=4096)
    U = run_batch(tb, tb.steps, "f32")
    prim = tb.prim()
    off = np.concatenate([[0], np.cumsum(tb.lengths)[:-1]])
    rng = np.random.default_rng(0)
    sample = list(rng.choice(4096, size=10, replace=False))
    sample += [int(np.argmin(tb.lengths)), int(np.argmax(tb.steps * tb.lengths))]
    worst = 0.0
    for b in sample:
        ref = oracle_tube(tb, b, tb.steps[b], prim, off)
        got = U[:, off[b]:off[b] + tb.lengths[b]]
        l1 = float(np.mean(np.abs(got[0] - ref[0])))
        worst = max(worst, l1)
        assert l1 <= 1e-5, (b, l1)
    print(f"4096 tubes: worst sampled density L1 vs FP64 oracle {worst:.2e}")


# ------------------------------------------------------------------- batched D1Q3

def run_batch_q3(tb, steps, precision, tuning=None, boundary="transmissive", prim=None):
    from paper_1504_07034_gb300.solver import BatchSolver
    s = BatchSolver(tb.lengths, tb.lam, gamma=tb.gamma, omega=tb.omega, boundary=boundary, precision=precision,
                    lattice="d1q3")
    if tuning:
        s.tuning = tuning
    s.set_state(torch.from_numpy(tb.prim() if prim is None else prim).cuda())
    s.run(steps)
    U = s.moments().cpu().numpy()
    f = s.get_distributions()
    assert tuple(f.shape) == (3, 3, tb.total_cells)
    s.close()
    return U


def oracle_tube_q3(tb, b, steps, prim_all, offsets, boundary="transmissive"):
    n = int(tb.lengths[b])
    o = oracle.Oracle(oracle.D1Q3, n, lam=float(tb.lam[b]), omega=tb.omega, gamma=tb.gamma,
                      bc=[(boundary, None)] * 2)
    fs, _ = o.run(o.init(o.prim_to_cons(prim_all[:, offsets[b]:offsets[b] + n])), int(steps))
    return o.moments(fs)


@pytest.mark.parametrize("tuning", [None, (128, 1, 8), (512, 2, 64)])
@pytest.mark.parametrize("boundary", ["transmissive", "periodic"])
def test_f64_batched_d1q3_matches_oracle_per_tube(tuning, boundary):
    """The rest-particle model (Section II.C) in the batched kernel: each tube as a lone D1Q3 tube."""
    tb = W.batched_tubes(seed=4, count=17, n_min=1, n_max=500, t_final=0.1, omega=0.9, lattice="d1q3")
    rng = np.random.default_rng(4)
    steps = rng.integers(0, 250, size=17)
    prim = tb.prim()
    if boundary == "periodic":
        tb.lam = tb.lam * 1.5
    U = run_batch_q3(tb, steps, "f64", tuning, boundary, prim)
    off = np.concatenate([[0], np.cumsum(tb.lengths)[:-1]])
    for b in range(len(tb.lengths)):
        ref = oracle_tube_q3(tb, b, steps[b], prim, off, boundary)
        got = U[:, off[b]:off[b] + tb.lengths[b]]
        err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref))
        assert np.all(err <= 1e-12), (b, tb.lengths[b], steps[b], err)


def test_f32_batched_d1q3_close_to_oracle():
    tb = W.batched_tubes(seed=5, count=9, n_min=50, n_max=2000, t_final=0.15, lattice="d1q3")
    U = run_batch_q3(tb, tb.steps, "f32", (256, 2, 16))
    off = np.concatenate([[0], np.cumsum(tb.lengths)[:-1]])
    prim = tb.prim()
    for b in range(len(tb.lengths)):
        ref = oracle_tube_q3(tb, b, tb.steps[b], prim, off)
        got = U[:, off[b]:off[b] + tb.lengths[b]]
        assert np.mean(np.abs(got[0] - ref[0])) <= 1e-6
