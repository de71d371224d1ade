"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bars (written here, derived in the design notes):
  * FP64 path: max |U_gpu - U_oracle| / max |U_oracle| per conserved field <= 1e-12
    (both sides evaluate the same expressions in the same order without FMA,
    so the expected difference is zero; 1e-12 leaves room for nothing else);
  * FP32 path: density L1 error against the FP64 oracle, cell-averaged, stated
    as a number and bounded (<= 1e-5 on the 2-D configurations).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()
    oracle.build()
    torch.cuda.init()


def solver(wl, precision, **kw):
    from paper_1504_07034_gb300.solver import Solver
    return Solver.from_workload(wl, precision=precision, **kw)


def run_gpu(wl, precision, steps=None, W0=None):
    s = solver(wl, precision)
    s.set_state(torch.from_numpy(wl.prim if W0 is None else W0).cuda(), primitive=True)
    s.step(wl.steps if steps is None else steps)
    U = s.moments(torch.float64).cpu().numpy()
    fs = s.get_distributions().double().cpu().numpy()
    s.close()
    return U, fs


def run_oracle(wl, steps=None):
    o = oracle.Oracle.from_workload(wl)
    fs, chk = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps if steps is None else steps)
    return o.moments(fs), fs, chk


def field_rel_err(a, b):
    K = a.shape[0]
    glob = np.max(np.abs(b))
    errs = []
    for k in range(K):
        scale = np.max(np.abs(b[k])) or glob
        errs.append(np.max(np.abs(a[k] - b[k])) / scale)
    return np.array(errs)


def l1_rho(a, b):
    return float(np.mean(np.abs(a[0] - b[0])))


# ------------------------------------------------------------------- small 2-D cases

BC_SETS = {
    "transmissive": [("transmissive", None)] * 4,
    "periodic": [("periodic", None)] * 4,
    "dirichlet_wall": [("dirichlet", (1.2, 0.8, 0.1, 1.0)), ("transmissive", None), ("wall", None),
                       ("dirichlet", (0.9, 0.5, -0.3, 0.8))],
    "walls_periodic_x": [("periodic", None), ("periodic", None), ("wall", None), ("wall", None)],
    "mixed": [("transmissive", None), ("dirichlet", (1.0, -0.3, 0.2, 0.7)), ("dirichlet", (0.8, 0.1, 0.4, 0.9)),
              ("transmissive", None)],
    # the halfway alternative of the free-slip wall, against a Dirichlet x side (corner resolution)
    # and against the on-node wall on the other y side
    "halfway_dirichlet": [("dirichlet", (1.2, 0.8, 0.1, 1.0)), ("transmissive", None), ("wall_halfway", None),
                          ("wall", None)],
    "halfway_periodic_x": [("periodic", None), ("periodic", None), ("wall_halfway", None), ("wall_halfway", None)],
}


def small_case(nx, ny, bcname, omega, steps=60, seed=0):
    wl = W.quadrant_riemann(seed, 8, steps=steps, omega=omega)   # states + lambda from a seeded draw
    q = wl.meta["quadrants"]
    dx = 1.0 / max(nx, ny)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    xc, yc = 0.5 * nx * dx, 0.5 * ny * dx
    prim = np.empty((4, ny, nx))
    for k in range(4):
        prim[k] = np.where(Y >= yc, np.where(X >= xc, q[1][k], q[2][k]), np.where(X >= xc, q[4][k], q[3][k]))
    bc = BC_SETS[bcname]
    if any(kind == "wall" for kind, _ in bc):
        prim[2, 0, :] = 0.0 if bc[2][0] == "wall" else prim[2, 0, :]
        prim[2, -1, :] = 0.0 if bc[3][0] == "wall" else prim[2, -1, :]
    # generous lambda: periodic wraps and Dirichlet sides add Riemann problems of their own
    lam = 1.6 * max([wl.lam] + [W.bouchut_speed(1.4, *st) for kind, st in bc if kind == "dirichlet"])
    return W.Workload2D(f"small_{bcname}", nx, ny, dx, 0.0, 0.0, prim, bc, lam, omega, steps)


@pytest.mark.parametrize("bcname", sorted(BC_SETS))
@pytest.mark.parametrize("shape", [(200, 70), (133, 129), (37, 261)])
@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_f64_matches_oracle_small_2d(bcname, shape, omega):
    nx, ny = shape
    if bcname in ("periodic", "walls_periodic_x", "halfway_periodic_x") and (nx % 2 or ny % 2):
        nx += nx % 2
        ny += ny % 2
    wl = small_case(nx, ny, bcname, omega)
    U_ref, fs_ref, _ = run_oracle(wl)
    U, fs = run_gpu(wl, "f64")
    assert np.all(field_rel_err(U, U_ref) <= F64_TOL), field_rel_err(U, U_ref)
    assert np.max(np.abs(fs - fs_ref)) <= F64_TOL * np.max(np.abs(fs_ref))


@pytest.mark.parametrize("bcname", ["transmissive", "dirichlet_wall", "periodic", "halfway_dirichlet"])
def test_f32_close_to_oracle_small_2d(bcname):
    wl = small_case(160, 96, bcname, 1.0, steps=100)
    U_ref, _, _ = run_oracle(wl)
    U, _ = run_gpu(wl, "f32")
    err = l1_rho(U, U_ref)
    assert err <= 2e-6, err


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (2, 2), (3, 5)])
@pytest.mark.parametrize("bcname", ["transmissive", "mixed"])
def test_f64_degenerate_grids(shape, bcname):
    nx, ny = shape
    wl = small_case(nx, ny, bcname, 1.3, steps=9)
    U_ref, _, _ = run_oracle(wl)
    U, _ = run_gpu(wl, "f64")
    assert np.all(field_rel_err(U, U_ref) <= F64_TOL)


def test_zero_steps_is_initial_equilibrium():
    wl = small_case(40, 30, "transmissive", 1.0, steps=0)
    U_ref, fs_ref, _ = run_oracle(wl, 0)
    U, fs = run_gpu(wl, "f64", 0)
    assert np.array_equal(fs, fs_ref)
    assert np.all(field_rel_err(U, U_ref) <= F64_TOL)


def test_graph_path_equals_single_steps():
    """lbrs_step(n) replays a captured graph for long runs and, in FP32, advances two steps per
    launch; it must equal n single steps bitwise."""
    wl = small_case(100, 64, "dirichlet_wall", 1.2, steps=0)
    a = solver(wl, "f32")
    b = solver(wl, "f32")
    W0 = torch.from_numpy(wl.prim).cuda()
    a.set_state(W0)
    b.set_state(W0)
    a.step(203)
    for _ in range(203):
        b.step(1)
    assert torch.equal(a.get_distributions(), b.get_distributions())
    assert a.step_count == b.step_count == 203
    a.close()
    b.close()


# ------------------------------------------------------------------- 1-D

@pytest.mark.parametrize("omega", [1.0, 0.7, 1.5])
def test_f64_sod_matches_oracle(omega):
    wl = W.sod(1000, omega=omega)
    U_ref, fs_ref, _ = run_oracle(wl)
    U, fs = run_gpu(wl, "f64")
    assert np.all(field_rel_err(U, U_ref) <= F64_TOL)


def test_f32_sod_l1():
    wl = W.sod(1000)
    U_ref, _, _ = run_oracle(wl)
    U, _ = run_gpu(wl, "f32")
    assert l1_rho(U, U_ref) <= 1e-5


@pytest.mark.parametrize("n", [1, 2, 257, 4099])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_f64_1d_sizes(n, bc):
    rng = np.random.default_rng(n)
    prim = np.array([rng.uniform(0.5, 2, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.5, 2, n)])
    state = (1.0, 0.2, 1.0)
    wl = W.Workload1D("rand1d", n, 1.0 / n, 0.0, prim, [(bc, state if bc == "dirichlet" else None)] * 2,
                      4.0, 1.2, 50)
    U_ref, _, _ = run_oracle(wl)
    U, _ = run_gpu(wl, "f64")
    assert np.all(field_rel_err(U, U_ref) <= F64_TOL)


# ------------------------------------------------------------------- full-size workloads

def test_full_size_quadrant_riemann_1024():
    """2-D four-quadrant Riemann problem, 1024 x 1024, 1000 steps: FP64 vs oracle and FP32 L1."""
    wl = W.quadrant_riemann(0, 1024, steps=1000)
    U_ref, _, chk = run_oracle(wl)
    assert chk["first_bad_step"] == -1
    U64, _ = run_gpu(wl, "f64")
    assert np.all(field_rel_err(U64, U_ref) <= F64_TOL), field_rel_err(U64, U_ref)
    U32, _ = run_gpu(wl, "f32")
    err = l1_rho(U32, U_ref)
    print(f"quadrant_riemann 1024^2 x 1000: FP32 density L1 vs FP64 oracle = {err:.3e}")
    assert err <= 1e-5


def test_full_size_oblique_shock_sampled():
    """Oblique shock reflection at its full 4096 x 1024 size, first 150 steps (the oracle's share)."""
    wl = W.oblique_shock_reflection(steps=150)
    U_ref, _, chk = run_oracle(wl)
    assert chk["first_bad_step"] == -1
    U64, _ = run_gpu(wl, "f64")
    assert np.all(field_rel_err(U64, U_ref) <= F64_TOL)
    U32, _ = run_gpu(wl, "f32")
    assert l1_rho(U32, U_ref) <= 1e-5


# ------------------------------------------------------------------- API behaviour

def test_moments_host_device_and_dtypes():
    wl = small_case(64, 48, "transmissive", 1.0, steps=20)
    s = solver(wl, "f64")
    s.set_state(wl.prim)                                   # host numpy input
    s.step(20)
    dev = s.moments(torch.float64)
    host = s.moments(out=torch.empty((4, 48, 64), dtype=torch.float64))
    f32 = s.moments(torch.float32)
    assert torch.equal(dev.cpu(), host)
    assert torch.equal(f32.cpu(), host.float())
    s.close()


def test_set_state_conserved_and_float32_input():
    wl = small_case(50, 40, "periodic", 1.0, steps=5)
    o = oracle.Oracle.from_workload(wl)
    U0 = o.prim_to_cons(wl.prim)
    s = solver(wl, "f64")
    s.set_state(torch.from_numpy(U0).cuda(), primitive=False)
    fs = s.get_distributions().cpu().numpy()
    assert np.max(np.abs(fs - o.init(U0))) <= 1e-15 * np.abs(fs).max()
    s.set_state(torch.from_numpy(wl.prim).float().cuda(), primitive=True)
    U = s.moments().cpu().numpy()
    assert np.max(np.abs(U - o.prim_to_cons(wl.prim.astype(np.float32).astype(np.float64)))) < 1e-14 * np.abs(U).max()
    s.close()


def test_checkpoint_resume_bitwise():
    wl = small_case(90, 60, "dirichlet_wall", 1.5, steps=0)
    a = solver(wl, "f32")
    a.set_state(torch.from_numpy(wl.prim).cuda())
    a.step(40)
    ck = a.get_distributions().cpu()
    a.step(70)
    end = a.get_distributions()
    b = solver(wl, "f32")
    b.set_distributions(ck, step=40)
    b.step(70)
    assert torch.equal(b.get_distributions(), end)
    assert b.step_count == 110
    a.close()
    b.close()


def test_diagnostics_match_oracle():
    wl = small_case(128, 96, "dirichlet_wall", 1.0, steps=80)
    o = oracle.Oracle.from_workload(wl)
    fs, _ = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps)
    tot_ref = o.totals(fs, wl.dx * wl.dx)
    s = solver(wl, "f64")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(wl.steps)
    d = s.diagnostics()
    assert d["status"] == "LBRS_OK"
    assert np.allclose(d["totals"], tot_ref, rtol=1e-12, atol=1e-15)
    Wp = o.cons_to_prim(o.moments(fs))
    assert d["min_rho"] == pytest.approx(Wp[0].min(), rel=1e-12)
    assert d["min_p"] == pytest.approx(Wp[3].min(), rel=1e-12)
    d2 = s.diagnostics()
    assert d2["totals"] == d["totals"]                 # fixed reduction order: bitwise repeatable
    s.close()


def test_subcharacteristic_violation_reported():
    wl = W.sod(400)
    wl.lam = 1.5                                       # below the post-shock u + a of about 2.19
    s = solver(wl, "f64")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(60)
    d = s.diagnostics()
    assert d["status"] in ("LBRS_ESUBCHAR", "LBRS_ENONPHYS")
    assert d["n_subchar"] > 0 or d["n_nonphysical"] > 0
    s.close()


def test_errors_state_and_arguments():
    from paper_1504_07034_gb300 import abi
    wl = small_case(16, 16, "transmissive", 1.0, steps=0)
    s = solver(wl, "f32")
    with pytest.raises(abi.LbrsError) as e:
        s.step(1)
    assert e.value.status == abi.LBRS_ESTATE
    s.set_state(torch.from_numpy(wl.prim).cuda())
    with pytest.raises(abi.LbrsError) as e:
        s.step(-1)
    assert e.value.status == abi.LBRS_EINVAL
    with pytest.raises(ValueError):
        s.set_state(torch.zeros(4, 3, 3, dtype=torch.float64, device="cuda"))
    s.close()


# ------------------------------------------------------------------- FP32 kernel variants

@pytest.mark.parametrize("bcname", sorted(BC_SETS))
@pytest.mark.parametrize("shape", [(200, 70), (36, 41), (516, 9), (4, 6), (130, 50)])
def test_f32_matches_oracle_every_boundary(bcname, shape):
    """FP32 path (vectorised kernel where nx % 4 == 0, scalar otherwise) close to the FP64 oracle."""
    nx, ny = shape
    if bcname in ("periodic", "walls_periodic_x", "halfway_periodic_x") and (nx % 2 or ny % 2):
        ny += ny % 2
    wl = small_case(nx, ny, bcname, 1.3, steps=60)
    U_ref, _, _ = run_oracle(wl)
    U, _ = run_gpu(wl, "f32")
    # normwise: FP32 rounding is relative to the size of the state, not of a
    # field that may sit near zero (rho v between walls)
    err = np.max(np.abs(U - U_ref), axis=tuple(range(1, U.ndim))) / np.max(np.abs(U_ref))
    assert np.all(err <= 2e-5), err


_VARIANT_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import workloads as W
from paper_1504_07034_gb300.solver import Solver
out = []
D = [("dirichlet", (1.0, 0.5, 0.1, 1.0)), ("dirichlet", (0.8, -0.2, 0.0, 0.9))]
T = ("transmissive", None)
P = ("periodic", None)
Wl = ("wall", None)
Hw = ("wall_halfway", None)
for bc in ([T] * 4, [P] * 4, D + [T, T], [T, D[1], Wl, D[0]], [P, P, Wl, Wl], [D[0], T, D[1], Wl], [P, P, Hw, Hw],
           [D[0], T, Hw, Wl]):
    wl = W.quadrant_riemann(1, 64, steps=50)
    for nx, ny in ((256, 48), (64, 48), (12, 48), (37, 29), (66, 17), (5, 3), (1, 9), (33, 1)):
        if bc[0] == P and nx % 2:
            nx += 1
        if bc[2] == P and ny % 2:
            ny += 1
        if Wl in (bc[2], bc[3]):
            ny = max(ny, 2)
        prim = np.ascontiguousarray(np.tile(wl.prim, (1, 1, 4))[:, :ny, :nx])
        if bc[2] == Wl:
            prim[2, 0, :] = 0.0
        if bc[3] == Wl:
            prim[2, -1, :] = 0.0
        s = Solver("d2q4", nx, ny, lam=1.6 * wl.lam, dx=1.0 / 64, bc=bc, precision="f32")
        s.set_state(torch.from_numpy(prim).cuda())
        s.step(51)
        out.append(s.get_distributions().cpu().numpy().ravel())
        out.append(s.step_record(7).cpu().numpy().ravel())      # recording steps: 3 pairs and a single
        out.append(s.get_distributions().cpu().numpy().ravel())
        s.close()
np.save(sys.argv[2], np.concatenate(out))
"""


def test_f32_kernel_variants_agree(tmp_path):
    """Scalar, vector-width and strided one-step kernels and the multi-step kernels compute the
    same steps.  The three- and two-steps-per-launch kernels run the scalar kernel's per-cell code
    (same loads, boundary resolution and collision helper), so they must agree bit for bit; the
    other variants up to FMA contraction.  Where nx % 4 == 0 lbrs_step takes three steps per
    launch (tensor copies of 40 x 20 boxes; with LBRS_F32_FUSE3=0 the two-step kernel's 36 x 18
    copies), elsewhere two (direct loads; everywhere with LBRS_F32_TMA=0).  51 steps: a graph
    (36 steps in threes, or 32 in twos), then the rest; then 7 recording steps (moments of every
    step, as the adjoint recompute takes them)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "variant.py"
    script.write_text(_VARIANT_SCRIPT)
    res = {}
    for v in ("0", "2", "4", "12", "14", "fused", "fused2", "fused_direct"):
        out = tmp_path / f"v{v}.npy"
        fused = v.startswith("fused")
        env = dict(os.environ, LBRS_F32_STEP_VARIANT="0" if fused else v, LBRS_F32_FUSE="1" if fused else "0",
                   LBRS_F32_TMA="0" if v == "fused_direct" else "1", LBRS_F32_FUSE3="1" if v == "fused" else "0")
        subprocess.run([sys.executable, str(script), root, str(out)], check=True, env=env, timeout=300)
        res[v] = np.load(out)
    scale = np.abs(res["0"]).max()
    for v in ("2", "4", "12", "14"):
        assert np.max(np.abs(res[v] - res["0"])) <= 1e-5 * scale, v
    for v in ("fused", "fused2", "fused_direct"):
        assert np.array_equal(res[v], res["0"]), (v, np.max(np.abs(res[v] - res["0"])) / scale)


def test_f32_three_steps_take_one_launch():
    """Where nx % 4 == 0 the FP32 path advances three steps with one launch of the three-step kernel
    (its tensor map accepted on this device); a grid it cannot tile takes more launches."""
    from paper_1504_07034_gb300.solver import Solver
    wl = W.quadrant_riemann(1, 64, steps=0)
    for nx, launches in ((256, 1), (66, 2)):
        prim = np.ascontiguousarray(np.tile(wl.prim, (1, 1, 5))[:, :, :nx])
        s = Solver("d2q4", nx, 64, lam=wl.lam, dx=1.0 / 64, bc=[("transmissive", None)] * 4, precision="f32")
        s.set_state(torch.from_numpy(prim).cuda())
        l0 = s.launch_count
        s.step(3)
        torch.cuda.synchronize()
        assert s.launch_count - l0 == launches, (nx, s.launch_count - l0)
        s.close()


# ------------------------------------------------------------------- periodic device checks

@pytest.mark.parametrize("every", [1, 5])
def test_periodic_checks_report_first_bad_step(every):
    from paper_1504_07034_gb300 import abi
    from paper_1504_07034_gb300.solver import Solver
    wl = W.sod(400)
    wl.lam = 1.5                                       # below the post-shock u + a of about 2.19
    o = oracle.Oracle.from_workload(wl)
    _, chk = o.run(o.init(o.prim_to_cons(wl.prim)), 60)
    first = chk["first_bad_step"]
    assert first >= 1
    s = Solver.from_workload(wl, precision="f64", diag_every=every)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(60)
    with pytest.raises(abi.LbrsError) as e:
        s.sync()
    assert e.value.status in (abi.LBRS_ESUBCHAR, abi.LBRS_ENONPHYS)
    expected = -(-first // every) * every              # first multiple of `every` at or after it
    assert s.first_bad_step() == expected
    s.set_state(torch.from_numpy(wl.prim).cuda())     # a new state clears the record
    assert s.first_bad_step() == -1
    s.close()


def test_periodic_checks_quiet_on_a_healthy_run():
    from paper_1504_07034_gb300.solver import Solver
    wl = W.quadrant_riemann(0, 256, steps=300)
    s = Solver.from_workload(wl, precision="f32", diag_every=10)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(wl.steps)
    s.sync()
    assert s.first_bad_step() == -1
    s.close()
