"""GPU parity of the y-slab path: several cut contexts equal one unsplit context.

One grid is split into 2, 3 or 5 y-slabs, each a context of liblbrs with cut y sides
(LBRS_BC_CUT, H ghost rows), all on this one GPU; the driver of
paper_1504_07034_gb300.slabs moves the exchanged rows between them with device
copies (lbrs_halo_export / lbrs_halo_import) on one stream, so no kernel ever waits
on another.  Bars:
  * FP64, FP32 and the moments-only form: the slabs' own rows equal the unsplit
    context's rows bit for bit (same kernels, same per-cell arithmetic);
  * FP64 additionally against the FP64 oracle, <= 1e-12 per field.
The cases cover the transmissive, periodic and wall + Dirichlet boundary sets,
tiled grids with a ragged edge (nx % 4 != 0 takes the direct-load two-step kernel,
nx % 4 == 0 the tensor-copy one), odd halo depths and step chunks that do not line
up with them.  The last test runs two processes on this GPU as gloo ranks (blocks
through host memory), the DistSlab path with the real library.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]

F64_TOL = 1e-12
CHUNKS = (1, 4, 7, 2, 17, 9)          # 40 steps


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_07034_gb300.build import build
    build()
    oracle.build()
    torch.cuda.init()


def _ragged(nx, ny, bc):
    wl = W.quadrant_riemann(3, 8, steps=40)
    q = wl.meta["quadrants"]
    dx = 1.0 / max(nx, ny)
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    prim = np.empty((4, ny, nx))
    for k in range(4):
        prim[k] = np.where(Y >= 0.5 * ny * dx, np.where(X >= 0.5 * nx * dx, q[1][k], q[2][k]),
                           np.where(X >= 0.5 * nx * dx, q[4][k], q[3][k]))
    if bc[2][0] == "wall":
        prim[2, 0, :] = 0.0
    lam = 1.6 * max([wl.lam] + [W.bouchut_speed(1.4, *st) for kind, st in bc if kind == "dirichlet"])
    return W.Workload2D("ragged", nx, ny, dx, 0.0, 0.0, prim, bc, lam, 1.0, 40)


CASES = {
    "transmissive": lambda: W.quadrant_riemann(2, 64, steps=40),
    "periodic": lambda: W.adjoint_pulses(seed=1, n=64, steps=40, width=0.1, pulses=3)[0],
    "walls_dirichlet": lambda: W.oblique_shock_reflection(nx=192, ny=48, steps=40),
    "ragged_dirichlet_wall": lambda: _ragged(202, 131, [("dirichlet", (1.2, 0.8, 0.1, 1.0)), ("transmissive", None),
                                                        ("wall", None), ("dirichlet", (0.9, 0.5, -0.3, 0.8))]),
    "ragged_periodic_x_walls": lambda: _ragged(133, 70, [("periodic", None), ("periodic", None), ("wall", None),
                                                         ("wall", None)]),
    "ragged_halfway_walls": lambda: _ragged(98, 61, [("dirichlet", (1.2, 0.8, 0.1, 1.0)), ("transmissive", None),
                                                     ("wall_halfway", None), ("wall_halfway", None)]),
}


def _solver(wl, precision, ny=None, bc=None):
    from paper_1504_07034_gb300.solver import Solver
    return Solver("d2q4", wl.nx, wl.ny if ny is None else ny, lam=wl.lam, dx=wl.dx,
                  bc=wl.bc if bc is None else bc, gamma=wl.gamma, omega=wl.omega, precision=precision)


def _unsplit(wl, precision, steps=40):
    s = _solver(wl, precision)
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(steps)
    U = s.moments(torch.float64).cpu().numpy()
    f = s.get_distributions().cpu().numpy() if precision in ("f64", "f32") else None
    s.close()
    return U, f


def _split(wl, precision, parts, halo, chunks=CHUNKS):
    from paper_1504_07034_gb300 import slabs
    bounds = slabs.slab_bounds(wl.ny, parts, halo)
    ss = []
    for r, (j0, j1) in enumerate(bounds):
        s = _solver(wl, precision, ny=j1 - j0, bc=slabs.slab_bc(wl.bc, r, parts, halo))
        s.set_state(torch.from_numpy(np.ascontiguousarray(wl.prim[:, j0:j1, :])).cuda())
        ss.append(s)
    run = slabs.LocalSlabs(ss, slabs.is_periodic_y(wl.bc))
    for n in chunks:
        run.step(n)
    U = np.concatenate([s.moments(torch.float64).cpu().numpy() for s in ss], axis=1)
    f = (np.concatenate([s.get_distributions().cpu().numpy() for s in ss], axis=2)
         if precision in ("f64", "f32") else None)
    diag = run.diagnostics()
    for s in ss:
        s.close()
    return U, f, diag


def _field_rel_err(a, b):
    return max(np.max(np.abs(a[k] - b[k])) / (np.max(np.abs(b[k])) or 1.0) for k in range(a.shape[0]))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("parts,halo", [(2, 2), (3, 2), (5, 3)])
@pytest.mark.parametrize("precision", ["f64", "f32", "f32u"])
def test_slabs_equal_unsplit_context(case, parts, halo, precision):
    if precision == "f32u" and "halfway" in case:
        pytest.skip("halfway walls are defined for the distribution forms")
    wl = CASES[case]()
    U_ref, f_ref = _unsplit(wl, precision)
    U, f, _ = _split(wl, precision, parts, halo)
    assert np.array_equal(U, U_ref), f"moments differ: max {np.max(np.abs(U - U_ref))}"
    if f_ref is not None:
        assert np.array_equal(f, f_ref)
    if precision == "f64":
        o = oracle.Oracle.from_workload(wl)
        fs, _ = o.run(o.init(o.prim_to_cons(wl.prim)), 40)
        assert _field_rel_err(U, o.moments(fs)) <= F64_TOL


def test_slab_diagnostics_add_up_to_the_grid():
    wl = CASES["walls_dirichlet"]()
    s = _solver(wl, "f64")
    s.set_state(torch.from_numpy(wl.prim).cuda())
    s.step(40)
    ref = s.diagnostics()
    s.close()
    _, _, d = _split(wl, "f64", 3, 2)
    assert np.allclose(d["totals"], ref["totals"], rtol=1e-13, atol=0)
    for key in ("min_rho", "min_p", "max_lambda_local", "n_nonphysical", "n_subchar", "status"):
        assert d[key] == ref[key], key


def test_slab_steps_need_imports():
    from paper_1504_07034_gb300 import abi, slabs
    wl = CASES["periodic"]()
    s0 = _solver(wl, "f32", ny=32, bc=slabs.slab_bc(wl.bc, 0, 2))
    s1 = _solver(wl, "f32", ny=32, bc=slabs.slab_bc(wl.bc, 1, 2))
    for s, rows in ((s0, slice(0, 32)), (s1, slice(32, 64))):
        s.set_state(torch.from_numpy(np.ascontiguousarray(wl.prim[:, rows, :])).cuda())
    assert s0.halo_size(2) == (2, 16 * 2 * 64 * 4)
    with pytest.raises(abi.LbrsError) as e:
        s0.step(1)                                  # no import since the state was set
    assert e.value.status == abi.LBRS_ESTATE
    run = slabs.LocalSlabs([s0, s1], True)
    run.exchange()
    with pytest.raises(abi.LbrsError):
        s0.step(3)                                  # beyond the two ghost rows
    s0.step(2)
    with pytest.raises(abi.LbrsError):
        s0.step(1)
    assert s0.step_count == 2
    s0.close()
    s1.close()


def test_slab_checkpoint_resume_bitwise():
    from paper_1504_07034_gb300 import slabs
    wl = CASES["transmissive"]()
    U_ref, _ = _unsplit(wl, "f32", steps=24)
    ss = []
    for r, (j0, j1) in enumerate(slabs.slab_bounds(wl.ny, 2)):
        s = _solver(wl, "f32", ny=j1 - j0, bc=slabs.slab_bc(wl.bc, r, 2))
        s.set_state(torch.from_numpy(np.ascontiguousarray(wl.prim[:, j0:j1, :])).cuda())
        ss.append(s)
    run = slabs.LocalSlabs(ss, False)
    run.step(10)
    blobs = [s.checkpoint() for s in ss]
    run.step(6)                                      # diverge, then resume from the blobs
    for s, b in zip(ss, blobs):
        s.restore(b)
    run.invalidate()
    run.step(14)
    U = np.concatenate([s.moments(torch.float64).cpu().numpy() for s in ss], axis=1)
    assert np.array_equal(U, U_ref)
    for s in ss:
        s.close()


def test_cut_configurations_refused_where_not_covered():
    from paper_1504_07034_gb300 import abi, slabs
    wl = CASES["periodic"]()
    bc = slabs.slab_bc(wl.bc, 0, 2)
    with pytest.raises(abi.LbrsError):
        _solver(wl, "f16neq", ny=32, bc=bc)
    with pytest.raises(abi.LbrsError):
        _solver(wl, "f32", ny=32, bc=[("cut", 2)] * 4)          # cuts on x sides
    with pytest.raises(abi.LbrsError):
        _solver(wl, "f32", ny=1, bc=bc)                           # fewer rows than ghost rows
    s = _solver(wl, "f32", ny=32, bc=bc)
    s.set_state(torch.from_numpy(np.ascontiguousarray(wl.prim[:, :32, :])).cuda())
    with pytest.raises(abi.LbrsError):
        s.set_obstacles(torch.zeros((32, 64), dtype=torch.uint8))
    with pytest.raises(abi.LbrsError):
        s.step_adaptive(1)
    with pytest.raises(abi.LbrsError):
        s.forward_checkpointed(4, 2)                              # steps without the neighbours' rows
    buf = s.halo_buffer(2)
    with pytest.raises(abi.LbrsError):
        s.halo_export(1, buf)                                     # not a y side
    s.close()


def test_poisoned_ghost_populations_stay_out_of_own_rows_and_checks():
    """Within H = 2 steps the own rows read, from the ghost rows beyond y-lo, only the
    populations moving up (q = 3, 4) and, beyond y-hi, only those moving down (q = 1, 2).
    Imports whose other populations are NaN must leave the own rows bit-identical to the
    unsplit run, and the periodic checks (diag_every = 2), which then meet NaN in the ghost
    rows, must flag nothing."""
    from paper_1504_07034_gb300 import slabs
    from paper_1504_07034_gb300.solver import Solver
    wl = CASES["walls_dirichlet"]()
    U_ref, _ = _unsplit(wl, "f32")
    bounds = slabs.slab_bounds(wl.ny, 3)
    ss = []
    for r, (j0, j1) in enumerate(bounds):
        s = Solver("d2q4", wl.nx, j1 - j0, lam=wl.lam, dx=wl.dx, bc=slabs.slab_bc(wl.bc, r, 3), gamma=wl.gamma,
                   omega=wl.omega, precision="f32", diag_every=2)
        s.set_state(torch.from_numpy(np.ascontiguousarray(wl.prim[:, j0:j1, :])).cuda())
        ss.append(s)
    for _ in range(20):
        blocks = {}
        for r, s in enumerate(ss):
            for side in (2, 3):
                if s.halo_size(side)[0]:
                    blocks[(r, side)] = s.halo_export(side, s.halo_buffer(side)).clone()
        for r, s in enumerate(ss):
            if (r - 1, 3) in blocks:
                b = blocks[(r - 1, 3)].clone()
                b[0:8] = float("nan")              # q = 1, 2 (moving down): never read across y-lo
                s.halo_import(2, b)
            if (r + 1, 2) in blocks:
                b = blocks[(r + 1, 2)].clone()
                b[8:16] = float("nan")             # q = 3, 4 (moving up): never read across y-hi
                s.halo_import(3, b)
        for s in ss:
            s.step(2)
    U = np.concatenate([s.moments(torch.float64).cpu().numpy() for s in ss], axis=1)
    assert np.array_equal(U, U_ref)
    for s in ss:
        s.sync()
        assert s.first_bad_step() == -1
        assert s.diagnostics()["status"] == "LBRS_OK"
        s.close()


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1504_07034_gb300 import slabs
        torch.cuda.set_device(0)
        wl = CASES["ragged_dirichlet_wall"]()
        j0, j1 = slabs.slab_bounds(wl.ny, world)[rank]
        s = _solver(wl, "f32", ny=j1 - j0, bc=slabs.slab_bc(wl.bc, rank, world))
        s.set_state(torch.from_numpy(np.ascontiguousarray(wl.prim[:, j0:j1, :])).cuda())
        run = slabs.DistSlab(s, rank, world, slabs.is_periodic_y(wl.bc))
        for n in CHUNKS:
            run.step(n)
        d = run.diagnostics()
        np.save(os.path.join(out_dir, f"U{rank}.npy"), s.moments(torch.float64).cpu().numpy())
        np.save(os.path.join(out_dir, f"tot{rank}.npy"), np.array(d["totals"] + [d["min_rho"], d["min_p"]]))
        s.close()
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu(tmp_path):
    """Two processes, one slab each, on this GPU; the blocks travel through host memory (gloo),
    so neither process's kernels wait on the other's."""
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    wl = CASES["ragged_dirichlet_wall"]()
    U_ref, _ = _unsplit(wl, "f32")
    U = np.concatenate([np.load(tmp_path / f"U{r}.npy") for r in range(2)], axis=1)
    assert np.array_equal(U, U_ref)
    t0, t1 = np.load(tmp_path / "tot0.npy"), np.load(tmp_path / "tot1.npy")
    assert np.array_equal(t0, t1)


# ---------------------------------------------------------------- the adjoint on slabs (reverse halo)

@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("parts,halo", [(2, 2), (3, 2), (3, 1)])
def test_slab_gradient_equals_unsplit_gradient(precision, parts, halo):
    """dL/dU0 on y-slabs of a periodic grid: forward recording with the state's rows exchanged every
    H steps, the recorded moments' rows exchanged once, the adjoint state's rows before every H
    adjoint steps.  The own rows equal the unsplit context's gradient bit for bit (same kernels,
    same per-cell arithmetic); FP64 also the oracle's (1e-10 per field)."""
    from paper_1504_07034_gb300 import slabs
    wl, target = W.adjoint_pulses(seed=3, n=64, steps=0, width=0.1, pulses=3)
    steps = 21
    o = oracle.Oracle.from_workload(wl)
    U0 = o.prim_to_cons(wl.prim)
    dt = torch.float64 if precision == "f64" else torch.float32
    one = _solver(wl, precision)
    loss_ref, (g_ref,) = slabs.LocalSlabs([one], True).gradient(
        [torch.from_numpy(U0).to("cuda", dt)], [torch.from_numpy(target).to("cuda", dt)], steps)
    g_ref = g_ref.cpu().numpy()
    one.close()
    ss, U0s, tgts = [], [], []
    for r, (j0, j1) in enumerate(slabs.slab_bounds(wl.ny, parts, halo)):
        ss.append(_solver(wl, precision, ny=j1 - j0, bc=slabs.slab_bc(wl.bc, r, parts, halo)))
        U0s.append(torch.from_numpy(np.ascontiguousarray(U0[:, j0:j1])).to("cuda", dt))
        tgts.append(torch.from_numpy(np.ascontiguousarray(target[j0:j1])).to("cuda", dt))
    loss, grads = slabs.LocalSlabs(ss, True).gradient(U0s, tgts, steps)
    g = np.concatenate([x.cpu().numpy() for x in grads], axis=1)
    assert np.array_equal(g, g_ref), np.max(np.abs(g - g_ref))
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    if precision == "f64":
        fsT, _ = o.run(o.init(U0), steps)
        dLdU = np.zeros_like(U0)
        dLdU[0] = (o.moments(fsT)[0] - target) * wl.dx * wl.dx
        g_or, _ = o.gradient(U0, steps, dLdU)
        assert _field_rel_err(g, g_or) <= 1e-10
    for s in ss:
        s.close()
