"""Pins of the oracle's boundary balance of a step (orc_boundary_flux).

Streaming (Section II.D) moves each post-collision population to x + c_q, and the collision keeps
the moments (Section II.A), so the totals after one step are the totals before plus what crosses
the sides inwards minus what crosses them outwards.  The pins: that identity against the oracle's
own step over every side kind and corner combination, both 2-D lattices and ragged grids; a
closed form for a uniform state on a grid of transmissive sides; zero on a periodic grid.
"""
import numpy as np
import pytest

import oracle

T = ("transmissive", None)
P = ("periodic", None)
W = ("wall", None)
H = ("wall_halfway", None)
D1 = ("dirichlet", (1.2, 0.8, 0.1, 1.0))
D2 = ("dirichlet", (0.9, -0.5, -0.3, 0.8))

SIDES = {
    "transmissive": [T, T, T, T],
    "periodic": [P, P, P, P],
    "dirichlet_wall": [D1, T, W, D2],
    "walls_periodic_x": [P, P, W, W],
    "halfway": [D1, T, H, W],
    "halfway_periodic_x": [P, P, H, H],
    "mixed": [T, D2, D1, T],
}


def _state(nx, ny, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 1.5, (ny, nx))
    u = rng.uniform(-0.4, 0.4, (ny, nx))
    v = rng.uniform(-0.4, 0.4, (ny, nx))
    p = rng.uniform(0.5, 1.5, (ny, nx))
    return np.stack([rho, u, v, p])


@pytest.mark.parametrize("name", sorted(SIDES))
@pytest.mark.parametrize("shape", [(12, 9), (7, 6), (1, 4), (5, 2)])
def test_one_step_changes_totals_by_the_balance(name, shape):
    nx, ny = shape
    bc = SIDES[name]
    if bc[0] == P and nx % 2:
        nx += 1
    if bc[2] == P and ny % 2:
        ny += 1
    W0 = _state(nx, ny, 1)
    if W in bc[2:] or H in bc[2:]:
        W0[2, 0, :] = 0.0
        W0[2, -1, :] = 0.0
    dx = 1.0 / max(nx, ny)
    o = oracle.Oracle(oracle.D2Q4, nx, ny, lam=4.0, omega=1.3, bc=bc, dx=dx)
    fs = o.init(o.prim_to_cons(W0))
    fs, _ = o.run(fs, 3)
    t0 = o.totals(fs, dx * dx)
    fin, fout = o.boundary_flux(fs, dx * dx)
    fs1, _ = o.run(fs, 1)
    t1 = o.totals(fs1, dx * dx)
    scale = np.max(np.abs(t0)) + np.max(np.abs(fin)) + np.max(np.abs(fout))
    assert np.all(np.abs((t1 - t0) - (fin - fout)) <= 1e-13 * scale), ((t1 - t0), fin - fout)
    if name == "periodic":
        assert not np.any(fin) and not np.any(fout)
    else:
        assert np.any(fin) and np.any(fout)


def test_scalar_lattice_balance():
    nx, ny, dx = 11, 8, 1.0 / 11
    rng = np.random.default_rng(4)
    u = rng.uniform(-0.5, 0.5, (1, ny, nx))
    bc = [("dirichlet", (0.3, -0.2, 0, 0)), T, T, ("dirichlet", (-0.1, 0.4, 0, 0))]   # profiles and clamps
    o = oracle.Oracle(oracle.D2Q4S, nx, ny, lam=2.0, omega=1.0, bc=bc, dx=dx)
    fs = o.init(u)
    t0 = o.totals(fs, dx * dx)
    fin, fout = o.boundary_flux(fs, dx * dx)
    t1 = o.totals(o.run(fs, 1)[0], dx * dx)
    assert abs((t1 - t0)[0] - (fin - fout)[0]) <= 1e-14 * (abs(t0[0]) + abs(fin[0]) + abs(fout[0]))


@pytest.mark.parametrize("shape", [(6, 4), (1, 5), (9, 1), (1, 1)])
def test_uniform_state_on_transmissive_sides(shape):
    """Every diagonal population leaves from the cells of one row and one column (nx + ny - 1 of them,
    the corner once) and the same number of cells pull it back from a clamped source of the same value:
    inflow = outflow = (nx + ny - 1) U_k dx^2 per field."""
    nx, ny = shape
    dx = 0.25
    W0 = np.broadcast_to(np.array([1.1, 0.3, -0.2, 0.9])[:, None, None], (4, ny, nx)).copy()
    o = oracle.Oracle(oracle.D2Q4, nx, ny, lam=3.0, bc=[T] * 4, dx=dx)
    U = o.prim_to_cons(W0)
    fin, fout = o.boundary_flux(o.init(U), dx * dx)
    want = (nx + ny - 1) * U[:, 0, 0] * dx * dx
    assert np.allclose(fin, want, rtol=1e-14, atol=0)
    assert np.allclose(fout, want, rtol=1e-14, atol=0)


def test_balance_rejects_what_it_does_not_cover():
    o1 = oracle.Oracle(oracle.D1Q2, 10, lam=2.0, bc=[T, T])
    with pytest.raises(ValueError):
        o1.boundary_flux(o1.init(np.ones((3, 10))), 0.1)
