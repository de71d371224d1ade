"""Domain decomposition of the D2Q4 step into y-slabs, checked on the CPU.

The multi-GPU design shards the grid into y-slabs; each step needs, per cut,
one row of post-collision populations from the neighbour (the pull at a row
reads rows j +- 1 only).  Here each slab is advanced by the FP64 oracle on its
own rows plus one halo row per cut, and after every step the halo rows are
refreshed from the neighbours: the result must equal the unsplit run bit for
bit.  The second test runs the same exchange between two gloo ranks with
send/recv (world size 2, 127.0.0.1).
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W


def slab_bounds(ny, parts):
    edges = np.linspace(0, ny, parts + 1).round().astype(int)
    return [(int(edges[r]), int(edges[r + 1])) for r in range(parts)]


def slab_oracle(wl, j0, j1, periodic_y):
    """Oracle for rows [j0, j1) plus a halo row on every side that is a cut."""
    lo_cut = periodic_y or j0 > 0
    hi_cut = periodic_y or j1 < wl.ny
    rows = (j1 - j0) + lo_cut + hi_cut
    bc = list(wl.bc)
    if lo_cut:
        bc[2] = ("transmissive", None)      # the halo row is overwritten every step
    if hi_cut:
        bc[3] = ("transmissive", None)
    o = oracle.Oracle(oracle.D2Q4, wl.nx, rows, lam=wl.lam, omega=wl.omega, gamma=wl.gamma, bc=bc)
    return o, int(lo_cut), int(hi_cut)


def decomposed_run(wl, fs0, parts, steps):
    periodic_y = wl.bc[2][0] == "periodic"
    bounds = slab_bounds(wl.ny, parts)
    slabs = []
    for j0, j1 in bounds:
        o, lo, hi = slab_oracle(wl, j0, j1, periodic_y)
        idx = [(j0 - 1) % wl.ny] * lo + list(range(j0, j1)) + [j1 % wl.ny] * hi
        slabs.append([o, lo, hi, fs0[:, :, idx, :].copy()])
    for _ in range(steps):
        for s in slabs:
            o = s[0]
            s[3], _, _ = o.collide(o.stream(s[3]))
        own = [s[3][:, :, s[1]:s[3].shape[2] - s[2], :] for s in slabs]
        for r, s in enumerate(slabs):                  # refresh the halo rows from the neighbours
            if s[1]:
                s[3][:, :, 0, :] = own[(r - 1) % parts][:, :, -1, :]
            if s[2]:
                s[3][:, :, -1, :] = own[(r + 1) % parts][:, :, 0, :]
    return np.concatenate([s[3][:, :, s[1]:s[3].shape[2] - s[2], :] for s in slabs], axis=2)


CASES = {
    "transmissive": lambda: W.quadrant_riemann(2, 48, steps=0),
    "periodic": lambda: W.adjoint_pulses(seed=1, n=48, steps=0, width=0.1, pulses=3)[0],
    "walls_dirichlet": lambda: W.oblique_shock_reflection(nx=96, ny=24, steps=0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("parts", [2, 3, 5])
def test_slabs_equal_unsplit_run_bitwise(case, parts):
    wl = CASES[case]()
    o = oracle.Oracle.from_workload(wl)
    fs0 = o.init(o.prim_to_cons(wl.prim))
    ref, _ = o.run(fs0, 40)
    got = decomposed_run(wl, fs0, parts, 40)
    assert np.array_equal(got, ref)


def _rank_main(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = CASES["periodic"]()
    o_full = oracle.Oracle.from_workload(wl)
    fs0 = o_full.init(o_full.prim_to_cons(wl.prim))
    j0, j1 = slab_bounds(wl.ny, world)[rank]
    o, lo, hi = slab_oracle(wl, j0, j1, periodic_y=True)
    idx = [(j0 - 1) % wl.ny] + list(range(j0, j1)) + [j1 % wl.ny]
    fs = fs0[:, :, idx, :].copy()
    up, down = (rank + 1) % world, (rank - 1) % world
    for _ in range(30):
        fs, _, _ = o.collide(o.stream(fs))
        first = torch.from_numpy(np.ascontiguousarray(fs[:, :, 1, :]))
        last = torch.from_numpy(np.ascontiguousarray(fs[:, :, -2, :]))
        from_down = torch.empty_like(first)
        from_up = torch.empty_like(first)
        # send my last own row up and my first own row down; receive the halos
        reqs = [dist.isend(last, up), dist.isend(first, down), dist.irecv(from_down, down), dist.irecv(from_up, up)]
        for r in reqs:
            r.wait()
        fs[:, :, 0, :] = from_down.numpy()
        fs[:, :, -1, :] = from_up.numpy()
    own = torch.from_numpy(np.ascontiguousarray(fs[:, :, 1:-1, :]))
    gathered = [torch.empty_like(own) for _ in range(world)] if rank == 0 else None
    sizes = [b - a for a, b in slab_bounds(wl.ny, world)]
    if rank == 0:
        parts = [own]
        for r in range(1, world):
            t = torch.empty((4, 4, sizes[r], wl.nx), dtype=own.dtype)
            dist.recv(t, r)
            parts.append(t)
        ref, _ = o_full.run(fs0, 30)
        ok = np.array_equal(torch.cat(parts, dim=2).numpy(), ref)
        with open(result_path, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    else:
        dist.send(own, 0)
    del gathered
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halos(tmp_path):
    import socket
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    result = tmp_path / "result.txt"
    mp.start_processes(_rank_main, args=(2, port, str(result)), nprocs=2, join=True, start_method="spawn")
    assert result.read_text() == "ok"
