"""The y-slab driver (paper_1504_07034_gb300.slabs) checked on the CPU.

The driver's host logic -- partition, neighbours, the order of the point-to-point
messages, stepping in chunks that an exchange covers, the reduction of the
diagnostics -- runs here on slabs stepped by the FP64 oracle with the library's cut
semantics: H ghost rows stored beyond each cut, the stored grid closed
transmissively there.  The ghost rows start as NaN, so any value of them that
reached an own row before an import replaced it would show.  Every case must
equal the unsplit oracle run bit for bit: within one process (LocalSlabs) and
between gloo ranks (DistSlab, world sizes 2 and 3, 127.0.0.1).  The adjoint on
slabs of a periodic grid (the reverse halo) must give the oracle's unsplit
gradient bit for bit as well.
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
from paper_1504_07034_gb300 import slabs


class OracleSlab:
    """Rows [j0, j1) of a workload's grid stepped by the oracle, with the library's cut sides."""

    def __init__(self, wl, j0, j1, sides):
        self.nx, self.ny = wl.nx, j1 - j0
        self.H = {s: (sides[s][1] if sides[s][0] == "cut" else 0) for s in (2, 3)}
        bc = [sides[0], sides[1]] + [("transmissive", None) if sides[s][0] == "cut" else sides[s] for s in (2, 3)]
        rows = self.ny + self.H[2] + self.H[3]
        self.o = oracle.Oracle(oracle.D2Q4, wl.nx, rows, lam=wl.lam, omega=wl.omega, gamma=wl.gamma, bc=bc,
                               dx=wl.dx)
        self.own_o = oracle.Oracle(oracle.D2Q4, wl.nx, self.ny, lam=wl.lam, omega=wl.omega, gamma=wl.gamma,
                                   bc=[("transmissive", None)] * 4, dx=wl.dx)
        self.fs = np.full((4, 4, rows, wl.nx), np.nan)
        self.left = {2: 0, 3: 0}
        self.dx = wl.dx
        # the adjoint interface: stored-layout buffers, the adjoint over the stored rows wrapped in y
        self.K, self.ny_store, self.row0 = 4, rows, self.H[2]
        self.store_grid = (rows, wl.nx)
        self.oa = oracle.Oracle(oracle.D2Q4, wl.nx, rows, lam=wl.lam, omega=wl.omega, gamma=wl.gamma,
                                bc=[("periodic", None)] * 4, dx=wl.dx)

    def set_own(self, fs_rows):
        self.fs[:, :, self.H[2]:self.H[2] + self.ny, :] = fs_rows
        self.left = {2: 0, 3: 0}

    def own(self):
        return self.fs[:, :, self.H[2]:self.H[2] + self.ny, :]

    # the Solver interface the driver uses
    def halo_size(self, side):
        return self.H[side], 16 * self.H[side] * self.nx * 8

    def halo_buffer(self, side, device=None):
        return torch.empty((16, self.H[side], self.nx), dtype=torch.float64, device=device or "cpu")

    def _own_rows(self, side):
        r0 = self.H[2] if side == 2 else self.H[2] + self.ny - self.H[3]
        return slice(r0, r0 + self.H[side])

    def _ghost_rows(self, side):
        r0 = 0 if side == 2 else self.H[2] + self.ny
        return slice(r0, r0 + self.H[side])

    def halo_export(self, side, out):
        assert self.H[side], "export across a side that is not a cut"
        block = self.fs[:, :, self._own_rows(side), :].reshape(16, self.H[side], self.nx)
        out.copy_(torch.from_numpy(np.ascontiguousarray(block)))
        return out

    def halo_import(self, side, block):
        assert self.H[side], "import across a side that is not a cut"
        self.fs[:, :, self._ghost_rows(side), :] = block.cpu().numpy().reshape(4, 4, self.H[side], self.nx)
        self.left[side] = self.H[side]

    def step(self, n):
        for side in (2, 3):
            if self.H[side]:
                assert n <= self.left[side], "stepping past what the last import covers"
                self.left[side] -= n
        for _ in range(n):
            self.fs, _, _ = self.o.collide(self.o.stream(self.fs))

    # adjoint interface (stored layout, torch CPU tensors)
    def _fields_tensor(self, n=None):
        return torch.zeros(((n,) if n is not None else ()) + (4,) + self.store_grid, dtype=torch.float64)

    def own_rows(self, t):
        return t[..., self.row0:self.row0 + self.ny, :]

    def rows_export(self, side, buf, out):
        b = buf.reshape(-1, self.ny_store, self.nx)
        r0 = self.H[2] if side == 2 else self.H[2] + self.ny - self.H[3]
        out.copy_(b[:, r0:r0 + self.H[side], :])
        return out

    def rows_import(self, side, buf, block):
        b = buf.view(-1, self.ny_store, self.nx)
        r0 = 0 if side == 2 else self.H[2] + self.ny
        b[:, r0:r0 + self.H[side], :] = block

    def set_state(self, U0, primitive=False):
        assert not primitive
        self.set_own(self.own_o.init(U0.numpy()))

    def step_record(self, n, h):
        for side in (2, 3):
            if self.H[side]:
                assert n <= self.left[side], "recording past what the last import covers"
                self.left[side] -= n
        for m in range(n):
            self.fs, U, _ = self.o.collide(self.o.stream(self.fs))
            h[m].copy_(torch.from_numpy(U))
        return h

    def vjp_loss(self, target):
        own = np.ascontiguousarray(self.own())
        r = self.own_o.moments(own)[0] - self.own_rows(target).numpy()
        cell = self.dx * self.dx
        g = torch.zeros((4, 4) + self.store_grid, dtype=torch.float64)
        self.own_rows(g)[:, 0] = torch.from_numpy(r * cell)
        return float(0.5 * np.sum(r * r) * cell), g

    def adjoint_step(self, U_next, g):
        return torch.from_numpy(self.oa.adjoint_step(U_next.numpy(), g.numpy()))

    def vjp_equilibrium(self, U0, g):
        return torch.from_numpy(self.oa.vjp_equilibrium(U0.numpy(), g.numpy()))

    def diagnostics(self):
        own = np.ascontiguousarray(self.own())
        U = self.own_o.moments(own)
        prim = self.own_o.cons_to_prim(U)
        return {"status": "LBRS_OK", "totals": list(self.own_o.totals(own, self.dx * self.dx)),
                "min_rho": float(prim[0].min()), "min_p": float(prim[3].min()),
                "max_lambda_local": 0.0, "n_nonphysical": 0, "n_subchar": 0}


CASES = {
    "transmissive": lambda: W.quadrant_riemann(2, 48, steps=0),
    "periodic": lambda: W.adjoint_pulses(seed=1, n=48, steps=0, width=0.1, pulses=3)[0],
    "walls_dirichlet": lambda: W.oblique_shock_reflection(nx=96, ny=24, steps=0),
}


def _unsplit(wl, steps):
    o = oracle.Oracle.from_workload(wl)
    fs0 = o.init(o.prim_to_cons(wl.prim))
    return fs0, o.run(fs0, steps)[0], o


def _make_slabs(wl, fs0, parts, halo):
    out = []
    for r, (j0, j1) in enumerate(slabs.slab_bounds(wl.ny, parts, halo)):
        s = OracleSlab(wl, j0, j1, slabs.slab_bc(wl.bc, r, parts, halo))
        s.set_own(fs0[:, :, j0:j1, :])
        out.append(s)
    return out


def test_partition_and_neighbours():
    assert slabs.slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slabs.slab_bounds(1024, 8)[-1] == (896, 1024)
    with pytest.raises(ValueError):
        slabs.slab_bounds(5, 3)                       # slabs thinner than two rows
    assert slabs.neighbours(0, 3, False) == (None, 1)
    assert slabs.neighbours(2, 3, False) == (1, None)
    assert slabs.neighbours(0, 3, True) == (2, 1)
    assert slabs.neighbours(1, 2, True) == (0, 0)
    assert slabs.neighbours(0, 1, True) == (None, None)
    bc = [("dirichlet", (1, 2, 0, 1)), ("transmissive", None), ("wall", None), ("dirichlet", (2, 1, 0, 1))]
    assert slabs.slab_bc(bc, 0, 3) == bc[:2] + [bc[2], ("cut", 2)]
    assert slabs.slab_bc(bc, 1, 3, 3) == bc[:2] + [("cut", 3), ("cut", 3)]
    assert slabs.slab_bc(bc, 2, 3) == bc[:2] + [("cut", 2), bc[3]]
    per = [("periodic", None)] * 4
    assert slabs.slab_bc(per, 0, 2) == per[:2] + [("cut", 2), ("cut", 2)]
    assert slabs.slab_bc(per, 0, 1) == per


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("parts,halo", [(2, 2), (3, 2), (5, 1), (3, 3)])
def test_local_slabs_equal_unsplit_run_bitwise(case, parts, halo):
    wl = CASES[case]()
    steps = 31
    fs0, ref, _ = _unsplit(wl, steps)
    ss = _make_slabs(wl, fs0, parts, halo)
    run = slabs.LocalSlabs(ss, slabs.is_periodic_y(wl.bc))
    for n in (1, 4, 7, 2, 17):                       # chunks that do not line up with the halo depth
        run.step(n)
    got = np.concatenate([s.own() for s in ss], axis=2)
    assert np.array_equal(got, ref)


def test_local_slabs_diagnostics_add_up():
    wl = CASES["walls_dirichlet"]()
    fs0, ref, o = _unsplit(wl, 12)
    ss = _make_slabs(wl, fs0, 3, 2)
    run = slabs.LocalSlabs(ss, False)
    run.step(12)
    d = run.diagnostics()
    tot = o.totals(ref, wl.dx * wl.dx)
    assert np.allclose(d["totals"], tot, rtol=1e-13, atol=0)
    prim = o.cons_to_prim(o.moments(ref))
    assert d["min_rho"] == prim[0].min() and d["min_p"] == prim[3].min()


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _rank_main(rank, world, port, case, result_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = CASES[case]()
        o = oracle.Oracle.from_workload(wl)
        fs0 = o.init(o.prim_to_cons(wl.prim))
        j0, j1 = slabs.slab_bounds(wl.ny, world)[rank]
        s = OracleSlab(wl, j0, j1, slabs.slab_bc(wl.bc, rank, world))
        s.set_own(fs0[:, :, j0:j1, :])
        run = slabs.DistSlab(s, rank, world, slabs.is_periodic_y(wl.bc))
        for n in (3, 1, 8, 5):
            run.step(n)
        d = run.diagnostics()
        np.save(os.path.join(result_dir, f"own{rank}.npy"), s.own())
        np.save(os.path.join(result_dir, f"diag{rank}.npy"),
                np.array([*d["totals"], d["min_rho"], d["min_p"], *s.diagnostics()["totals"],
                          s.diagnostics()["min_rho"], s.diagnostics()["min_p"]]))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [(2, "periodic"), (3, "walls_dirichlet"), (3, "periodic")])
def test_gloo_ranks_equal_unsplit_run_bitwise(tmp_path, world, case):
    mp.start_processes(_rank_main, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    wl = CASES[case]()
    _, ref, _ = _unsplit(wl, 17)
    got = np.concatenate([np.load(tmp_path / f"own{r}.npy") for r in range(world)], axis=2)
    assert np.array_equal(got, ref)
    diag = [np.load(tmp_path / f"diag{r}.npy") for r in range(world)]
    for d in diag:                                     # every rank holds the reduced values
        assert np.array_equal(d[:6], diag[0][:6])
    local = np.array([d[6:] for d in diag])
    assert np.array_equal(diag[0][:4], local[:, :4].sum(axis=0)) or np.allclose(
        diag[0][:4], local[:, :4].sum(axis=0), rtol=1e-15, atol=0)
    assert diag[0][4] == local[:, 4].min() and diag[0][5] == local[:, 5].min()


# ---------------------------------------------------------------- the adjoint on slabs

def _gradient_case():
    wl, target = W.adjoint_pulses(seed=2, n=40, steps=0, width=0.1, pulses=3)
    o = oracle.Oracle.from_workload(wl)
    U0 = o.prim_to_cons(wl.prim)
    return wl, target, o, U0


def _oracle_gradient(steps):
    wl, target, o, U0 = _gradient_case()
    fsT, _ = o.run(o.init(U0), steps)
    cell = wl.dx * wl.dx
    r = o.moments(fsT)[0] - target
    dLdU = np.zeros_like(U0)
    dLdU[0] = r * cell
    grad, _ = o.gradient(U0, steps, dLdU)
    return float(0.5 * np.sum(r * r) * cell), grad


@pytest.mark.parametrize("parts,halo", [(2, 2), (3, 1), (4, 3)])
def test_local_slab_gradient_equals_unsplit_oracle_gradient(parts, halo):
    steps = 13
    wl, target, _, U0 = _gradient_case()
    ss, U0s, tgts = [], [], []
    for r, (j0, j1) in enumerate(slabs.slab_bounds(wl.ny, parts, halo)):
        ss.append(OracleSlab(wl, j0, j1, slabs.slab_bc(wl.bc, r, parts, halo)))
        U0s.append(torch.from_numpy(np.ascontiguousarray(U0[:, j0:j1])))
        tgts.append(torch.from_numpy(np.ascontiguousarray(target[j0:j1])))
    loss, grads = slabs.LocalSlabs(ss, True).gradient(U0s, tgts, steps)
    loss_ref, grad_ref = _oracle_gradient(steps)
    assert loss == pytest.approx(loss_ref, rel=1e-13)
    assert np.array_equal(np.concatenate([g.numpy() for g in grads], axis=1), grad_ref)


def _grad_rank_main(rank, world, port, result_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, target, _, U0 = _gradient_case()
        j0, j1 = slabs.slab_bounds(wl.ny, world)[rank]
        s = OracleSlab(wl, j0, j1, slabs.slab_bc(wl.bc, rank, world))
        run = slabs.DistSlab(s, rank, world, True)
        loss, (g,) = run.gradient([torch.from_numpy(np.ascontiguousarray(U0[:, j0:j1]))],
                                  [torch.from_numpy(np.ascontiguousarray(target[j0:j1]))], 11)
        np.save(os.path.join(result_dir, f"grad{rank}.npy"), g.numpy())
        np.save(os.path.join(result_dir, f"loss{rank}.npy"), np.array([loss]))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gradient_equals_unsplit_oracle_gradient(tmp_path, world):
    mp.start_processes(_grad_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    loss_ref, grad_ref = _oracle_gradient(11)
    got = np.concatenate([np.load(tmp_path / f"grad{r}.npy") for r in range(world)], axis=1)
    assert np.array_equal(got, grad_ref)
    for r in range(world):
        assert float(np.load(tmp_path / f"loss{r}.npy")[0]) == pytest.approx(loss_ref, rel=1e-13)


@pytest.mark.timeout(120)
def test_a_single_uncut_slab_steps_and_differentiates():
    """One slab of a periodic grid has no cuts: stepping and the gradient run without
    exchanges (and terminate) and equal the plain run."""
    steps = 9
    wl, target, _, U0 = _gradient_case()
    s = OracleSlab(wl, 0, wl.ny, slabs.slab_bc(wl.bc, 0, 1))
    run = slabs.LocalSlabs([s], True)
    loss, (g,) = run.gradient([torch.from_numpy(U0)], [torch.from_numpy(target)], steps)
    loss_ref, grad_ref = _oracle_gradient(steps)
    assert np.array_equal(g.numpy(), grad_ref)
    assert loss == loss_ref
    run.invalidate()
    run.step(5)

