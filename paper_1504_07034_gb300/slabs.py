"""Y-slab decomposition of one D2Q4 grid: one solver per slab, halo rows exchanged at the cuts.

The pull of the multi-D update (Section II.D) reads, for row j, the rows j - 1 and j + 1
only.  A grid split into y-slabs therefore needs, at each cut and each step, the row of the
neighbouring slab next to the cut.  Each slab is an ordinary ``Solver`` whose y sides at the
cuts are of kind ("cut", H): the library stores H ghost rows beyond such a side, and after
one import of the neighbour's H rows (``lbrs_halo_import``) the slab can take up to H steps
with its own rows equal, bit for bit, to the same rows of the unsplit grid.

This module
  * partitions the rows (``slab_bounds``) and gives each slab its boundary sides (``slab_bc``);
  * pairs the neighbours (``neighbours``; a periodic y axis wraps around);
  * moves the exchanged blocks: ``LocalSlabs`` for several slabs in one process (device copies
    on the solvers' stream, e.g. several slabs on one GPU), ``DistSlab`` for one slab per rank
    with ``torch.distributed`` point-to-point calls (NCCL between GPUs; with gloo the blocks go
    through host memory);
  * reduces the slabs' diagnostics: FP64 sums of the totals and counts, minima of rho and p,
    maximum of the local bound (``combine_diagnostics`` / ``DistSlab.diagnostics``);
  * runs the adjoint on slabs of a periodic grid (``gradient``): the transpose of the streaming
    pulls, for row j, from rows j - 1 and j + 1 as the forward step does, so the same halo runs
    the other way -- before every H adjoint steps each slab imports the neighbours' rows of the
    adjoint state dL/df*, and once after the forward run those of every recorded moment field.

A solver here is anything with ``halo_size``, ``halo_buffer``, ``halo_export``,
``halo_import``, ``step`` and ``diagnostics`` as ``paper_1504_07034_gb300.solver.Solver``
has them.  No arithmetic of the method lives in this file.
"""
from __future__ import annotations

from contextlib import nullcontext
from typing import Sequence

Y_LO, Y_HI = 2, 3
DEFAULT_HALO_ROWS = 2
_TAG_UP, _TAG_DOWN = 17, 18     # a y-hi block travels up to the upper neighbour, a y-lo block down


def slab_bounds(ny: int, parts: int, min_rows: int = DEFAULT_HALO_ROWS) -> list[tuple[int, int]]:
    """Rows [j0, j1) of each of `parts` slabs, sizes differing by at most one row."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    base, extra = divmod(ny, parts)
    if base < min_rows:
        raise ValueError(f"{ny} rows cannot give {parts} slabs of at least {min_rows} rows")
    out, j = [], 0
    for r in range(parts):
        n = base + (1 if r < extra else 0)
        out.append((j, j + n))
        j += n
    return out


def is_periodic_y(bc: Sequence) -> bool:
    return bc[Y_LO][0] == "periodic"


def neighbours(rank: int, parts: int, periodic_y: bool) -> tuple[int | None, int | None]:
    """(lower, upper) slab of slab `rank`; None where the slab side is a side of the grid."""
    if parts == 1:
        return None, None
    lower = rank - 1 if rank > 0 else (parts - 1 if periodic_y else None)
    upper = rank + 1 if rank < parts - 1 else (0 if periodic_y else None)
    return lower, upper


def slab_bc(bc: Sequence, rank: int, parts: int, halo_rows: int = DEFAULT_HALO_ROWS) -> list:
    """Boundary sides of slab `rank`: the grid's x sides, and per y side either the grid's side
    or a cut with `halo_rows` ghost rows."""
    lower, upper = neighbours(rank, parts, is_periodic_y(bc))
    out = list(bc[:2])
    out.append(("cut", halo_rows) if lower is not None else bc[Y_LO])
    out.append(("cut", halo_rows) if upper is not None else bc[Y_HI])
    return out


def combine_diagnostics(parts: Sequence[dict]) -> dict:
    """The grid's diagnostics from its slabs' (dicts as Solver.diagnostics returns them)."""
    K = len(parts[0]["totals"])
    tot = [sum(p["totals"][k] for p in parts) for k in range(K)]
    nbad = sum(p["n_nonphysical"] for p in parts)
    nsub = sum(p["n_subchar"] for p in parts)
    status = "LBRS_ENONPHYS" if nbad else ("LBRS_ESUBCHAR" if nsub else "LBRS_OK")
    return {"status": status, "totals": tot, "min_rho": min(p["min_rho"] for p in parts),
            "min_p": min(p["min_p"] for p in parts),
            "max_lambda_local": max(p["max_lambda_local"] for p in parts),
            "n_nonphysical": nbad, "n_subchar": nsub}


class _Stepping:
    """Steps in chunks that the last exchange covers, exchanging when it is used up."""

    halo_rows: int
    left: int

    def _covered(self) -> int:
        """Steps one exchange covers: the ghost rows of the cuts; without cuts, any number."""
        return self.halo_rows if self.halo_rows else 1 << 62

    def exchange(self):
        raise NotImplementedError

    def _step_all(self, n: int):
        raise NotImplementedError

    def step(self, n: int):
        while n > 0:
            if self.left == 0:
                self.exchange()
            m = min(self.left, n)
            self._step_all(m)
            self.left -= m
            n -= m

    def invalidate(self):
        """Call after a state was set on the solvers: the next step exchanges first (slabs
        without cuts need no exchange)."""
        self.left = 0 if self.halo_rows else self._covered()

    # ------------------------------------------------------------ the adjoint (periodic grids)
    def _locals(self) -> list:
        raise NotImplementedError

    def exchange_rows(self, bufs):
        """The ghost rows of stored-layout tensors (one per local slab, any number of planes)
        from the neighbours' own rows."""
        raise NotImplementedError

    def _sum(self, x: float) -> float:
        return x

    def gradient(self, U0s, targets, steps: int):
        """Loss L = sum over the grid of 1/2 (rho(T) - target)^2 dx^2 after `steps` steps from the
        conserved initial fields, and dL/dU0, on slabs of a periodic grid.  U0s, targets: per local
        slab its own rows ((K, ny, nx) and (ny, nx) tensors on its device).  Returns (L, [dL/dU0 of
        each local slab's own rows]).  The forward run records every step's moments (memory:
        steps x K fields per slab); the backward sweeps them with the adjoint step."""
        import torch
        sv = self._locals()
        H = self.halo_rows
        U0st = []
        for s, U0 in zip(sv, U0s):
            t = s._fields_tensor()
            t.zero_()
            s.own_rows(t).copy_(U0)
            U0st.append(t)
        self.exchange_rows(U0st)
        for s, U0 in zip(sv, U0s):
            s.set_state(U0, primitive=False)
        self.invalidate()
        hists = [s._fields_tensor(steps) for s in sv]
        t = 0
        while t < steps:
            if self.left == 0:
                self.exchange()
            m = min(self.left, steps - t)
            for s, h in zip(sv, hists):
                s.step_record(m, h[t:t + m])
            self.left -= m
            t += m
        self.exchange_rows(hists)
        losses, g = [], []
        for s, tgt in zip(sv, targets):
            tt = torch.zeros(s.store_grid, dtype=tgt.dtype, device=tgt.device)
            s.own_rows(tt).copy_(tgt)
            loss, gT = s.vjp_loss(tt)
            losses.append(loss)
            g.append(gT)
        loss = self._sum(sum(losses))
        t = steps
        while t > 0:
            self.exchange_rows(g)
            m = min(H, t) if H else t
            for _ in range(m):
                t -= 1
                g = [s.adjoint_step(h[t], gi) for s, h, gi in zip(sv, hists, g)]
        return loss, [s.own_rows(s.vjp_equilibrium(u, gi)) for s, u, gi in zip(sv, U0st, g)]


class LocalSlabs(_Stepping):
    """Slabs of one grid held in one process (their solvers may share one GPU).  The blocks
    move by device copies on the solvers' streams, in stream order; all solvers should use
    the same stream."""

    def __init__(self, solvers: Sequence, periodic_y: bool):
        self.solvers = list(solvers)
        self.periodic_y = periodic_y
        parts = len(self.solvers)
        self.nb = [neighbours(r, parts, periodic_y) for r in range(parts)]
        rows = {s.halo_size(side)[0] for s in self.solvers for side in (Y_LO, Y_HI)} - {0}
        if len(rows) > 1:
            raise ValueError("all cuts of one grid need the same number of ghost rows")
        self.halo_rows = rows.pop() if rows else 0
        self.blocks = {}
        for r, (lo, up) in enumerate(self.nb):
            if lo is not None:
                self.blocks[(r, Y_LO)] = self.solvers[r].halo_buffer(Y_LO)
            if up is not None:
                self.blocks[(r, Y_HI)] = self.solvers[r].halo_buffer(Y_HI)
        self.left = 0 if self.halo_rows else self._covered()

    def exchange(self):
        for (r, side), buf in self.blocks.items():
            self.solvers[r].halo_export(side, buf)
        for r, (lo, up) in enumerate(self.nb):
            if lo is not None:
                self.solvers[r].halo_import(Y_LO, self.blocks[(lo, Y_HI)])
            if up is not None:
                self.solvers[r].halo_import(Y_HI, self.blocks[(up, Y_LO)])
        self.left = self._covered()

    def _step_all(self, n: int):
        for s in self.solvers:
            s.step(n)

    def _locals(self) -> list:
        return self.solvers

    def exchange_rows(self, bufs):
        import torch
        blocks = {}
        for r, (lo, up) in enumerate(self.nb):
            s, b = self.solvers[r], bufs[r]
            planes = b.numel() // (s.ny_store * s.nx)
            for side, peer in ((Y_LO, lo), (Y_HI, up)):
                if peer is not None:
                    out = torch.empty((planes, s.halo_size(side)[0], s.nx), dtype=b.dtype, device=b.device)
                    blocks[(r, side)] = s.rows_export(side, b, out)
        for r, (lo, up) in enumerate(self.nb):
            if lo is not None:
                self.solvers[r].rows_import(Y_LO, bufs[r], blocks[(lo, Y_HI)])
            if up is not None:
                self.solvers[r].rows_import(Y_HI, bufs[r], blocks[(up, Y_LO)])

    def diagnostics(self) -> dict:
        return combine_diagnostics([s.diagnostics() for s in self.solvers])


class DistSlab(_Stepping):
    """This rank's slab of a grid split over the ranks of a torch.distributed group.

    Every exchange posts, in this order, the send of the y-hi block to the upper neighbour,
    the send of the y-lo block to the lower one, the receive from the lower neighbour (its
    y-hi block, into our y-lo ghost rows) and the receive from the upper one; with two ranks
    on a periodic axis both neighbours are the same rank, and this order pairs the messages
    by position (NCCL) as well as by tag (gloo).  With the NCCL backend the blocks stay on the
    GPU and the point-to-point calls are ordered with the solver's stream; with another
    backend they go through host memory.
    """

    def __init__(self, solver, rank: int, world: int, periodic_y: bool, group=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.solver = solver
        self.rank, self.world, self.group = rank, world, group
        self.lower, self.upper = neighbours(rank, world, periodic_y)
        self.halo_rows = max(solver.halo_size(Y_LO)[0], solver.halo_size(Y_HI)[0])
        on_gpu = dist.get_backend(group) == "nccl"
        dev = None if on_gpu else "cpu"
        self.stream = getattr(solver, "stream", None) if on_gpu else None
        self.send, self.recv = {}, {}
        for side, peer in ((Y_LO, self.lower), (Y_HI, self.upper)):
            if peer is not None:
                self.send[side] = solver.halo_buffer(side, device=dev)
                self.recv[side] = solver.halo_buffer(side, device=dev)
        self.left = 0 if self.halo_rows else self._covered()
        self._torch = torch

    def exchange(self):
        ctx = self._torch.cuda.stream(self.stream) if self.stream is not None else nullcontext()
        with ctx:
            for side, buf in self.send.items():
                self.solver.halo_export(side, buf)
            self._p2p(self.send, self.recv)
            for side, buf in self.recv.items():
                self.solver.halo_import(side, buf)
        self.left = self._covered()

    def _step_all(self, n: int):
        self.solver.step(n)

    def _locals(self) -> list:
        return [self.solver]

    def _p2p(self, send: dict, recv: dict):
        """Blocks of the y-hi and y-lo sides out, the neighbours' in, in the order of _ops."""
        dist, ops = self.dist, []
        if self.upper is not None:
            ops.append(dist.P2POp(dist.isend, send[Y_HI], self.upper, self.group, _TAG_UP))
        if self.lower is not None:
            ops.append(dist.P2POp(dist.isend, send[Y_LO], self.lower, self.group, _TAG_DOWN))
        if self.lower is not None:
            ops.append(dist.P2POp(dist.irecv, recv[Y_LO], self.lower, self.group, _TAG_UP))
        if self.upper is not None:
            ops.append(dist.P2POp(dist.irecv, recv[Y_HI], self.upper, self.group, _TAG_DOWN))
        for work in dist.batch_isend_irecv(ops):
            work.wait()

    def exchange_rows(self, bufs):
        torch, s = self._torch, self.solver
        (b,) = bufs
        planes = b.numel() // (s.ny_store * s.nx)
        dev = b.device if self.dist.get_backend(self.group) == "nccl" else "cpu"
        ctx = torch.cuda.stream(self.stream) if self.stream is not None else nullcontext()
        with ctx:
            send, recv = {}, {}
            for side, peer in ((Y_LO, self.lower), (Y_HI, self.upper)):
                if peer is not None:
                    shape = (planes, s.halo_size(side)[0], s.nx)
                    send[side] = s.rows_export(side, b, torch.empty(shape, dtype=b.dtype, device=dev))
                    recv[side] = torch.empty(shape, dtype=b.dtype, device=dev)
            self._p2p(send, recv)
            for side, block in recv.items():
                s.rows_import(side, b, block)

    def _sum(self, x: float) -> float:
        torch, dist = self._torch, self.dist
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return float(t.item())

    def diagnostics(self) -> dict:
        """The grid's diagnostics: this slab's, reduced over the group in FP64."""
        torch, dist = self._torch, self.dist
        d = self.solver.diagnostics()
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        K = len(d["totals"])
        sums = torch.tensor([*d["totals"], float(d["n_nonphysical"]), float(d["n_subchar"])],
                            dtype=torch.float64, device=dev)
        maxes = torch.tensor([-d["min_rho"], -d["min_p"], d["max_lambda_local"]], dtype=torch.float64, device=dev)
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=self.group)
        dist.all_reduce(maxes, op=dist.ReduceOp.MAX, group=self.group)
        s, m = sums.tolist(), maxes.tolist()
        nbad, nsub = int(s[K]), int(s[K + 1])
        status = "LBRS_ENONPHYS" if nbad else ("LBRS_ESUBCHAR" if nsub else "LBRS_OK")
        return {"status": status, "totals": s[:K], "min_rho": -m[0], "min_p": -m[1], "max_lambda_local": m[2],
                "n_nonphysical": nbad, "n_subchar": nsub}

    def first_bad_step(self) -> int:
        """The earliest step any slab's periodic device checks flagged (-1 if none)."""
        torch, dist = self._torch, self.dist
        step = self.solver.first_bad_step()
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([step if step >= 0 else 1 << 62], dtype=torch.int64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        v = int(t.item())
        return -1 if v == 1 << 62 else v
