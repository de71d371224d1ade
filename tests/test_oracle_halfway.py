"""Pins of the oracle's halfway free-slip wall (the flag alternative of the Section II.E wall).

The halfway wall reflects specularly at the plane half a cell beyond the wall row.  So
a domain closed by such walls on both y sides must evolve exactly as the lower half of
a periodic domain of twice the height whose upper half holds the mirror image (rows
reversed, populations f1 <-> f4 and f2 <-> f3 exchanged, rho v negated): the periodic
run knows nothing of walls, so this pins the relation's neighbour, population and sign
independently of how the oracle writes it.  The comparison holds to round-off (1e-13 per
field, about 1e-15 measured over 40 steps), not bit for bit: the moments are summed in q
order, which the mirror reverses.  Further pins: with periodic x
sides the walls conserve mass, x momentum and energy to round-off and reverse the y
momentum they absorb, and a uniform flow along the walls stays uniform.
"""
import numpy as np
import pytest

import oracle

GAMMA = 1.4


def _fields(nx, ny, seed, vy=0.0):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid((np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx, indexing="ij")
    w = np.empty((4, ny, nx))
    w[0] = 1.0 + 0.2 * np.sin(2 * np.pi * (x + rng.uniform())) * np.cos(np.pi * (y + rng.uniform()))
    w[1] = 0.3 + 0.2 * np.cos(2 * np.pi * (x + y + rng.uniform()))
    w[2] = vy + 0.2 * np.sin(2 * np.pi * (2 * x + rng.uniform())) * np.sin(np.pi * y)
    w[3] = 1.0 + 0.3 * np.cos(2 * np.pi * (x - y + rng.uniform())) ** 2
    return w


def _mirror_up(fs):
    """fs[q, k, j, i] -> the mirror image in y: rows reversed, q -> 3 - q, field 2 negated."""
    m = fs[::-1, :, ::-1, :].copy()
    m[:, 2] *= -1.0
    return m


X_SIDES = {
    "periodic": [("periodic", None), ("periodic", None)],
    "transmissive": [("transmissive", None), ("transmissive", None)],
    "inflow_outflow": [("dirichlet", (1.1, 0.6, 0.0, 1.0)), ("transmissive", None)],   # v = 0: mirror-symmetric
}


@pytest.mark.parametrize("xs", sorted(X_SIDES))
@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_walled_domain_is_half_of_the_mirror_doubled_periodic_domain(xs, omega):
    nx, ny, steps, lam = 24, 10, 40, 4.0
    walled = oracle.Oracle(oracle.D2Q4, nx, ny, lam=lam, omega=omega, gamma=GAMMA,
                           bc=X_SIDES[xs] + [("wall_halfway", None)] * 2)
    doubled = oracle.Oracle(oracle.D2Q4, nx, 2 * ny, lam=lam, omega=omega, gamma=GAMMA,
                            bc=X_SIDES[xs] + [("periodic", None)] * 2)
    fs = walled.init(walled.prim_to_cons(_fields(nx, ny, 3)))
    fd = np.concatenate([fs, _mirror_up(fs)], axis=2)
    a, _ = walled.run(fs, steps)
    b, _ = doubled.run(fd, steps)
    for k in range(4):
        scale = np.max(np.abs(b[:, k]))
        assert np.max(np.abs(a[:, k] - b[:, k, :ny, :])) <= 1e-13 * scale, k
        assert np.max(np.abs(_mirror_up(a)[:, k] - b[:, k, ny:, :])) <= 1e-13 * scale, k


def test_walls_conserve_mass_x_momentum_energy():
    nx, ny = 32, 12
    o = oracle.Oracle(oracle.D2Q4, nx, ny, lam=4.0, omega=1.3, gamma=GAMMA,
                      bc=[("periodic", None)] * 2 + [("wall_halfway", None)] * 2)
    fs0 = o.init(o.prim_to_cons(_fields(nx, ny, 5, vy=0.1)))
    t0 = o.totals(fs0, 1.0)
    fs, _ = o.run(fs0, 200)
    t1 = o.totals(fs, 1.0)
    for k in (0, 1, 3):
        assert abs(t1[k] - t0[k]) <= 1e-12 * abs(t0[k])


def test_uniform_flow_along_the_walls_stays_uniform():
    nx, ny = 16, 8
    o = oracle.Oracle(oracle.D2Q4, nx, ny, lam=4.0, omega=1.5, gamma=GAMMA,
                      bc=[("periodic", None)] * 2 + [("wall_halfway", None)] * 2)
    w = np.empty((4, ny, nx))
    w[0], w[1], w[2], w[3] = 1.2, 0.7, 0.0, 0.9
    fs0 = o.init(o.prim_to_cons(w))
    fs, _ = o.run(fs0, 100)
    assert np.max(np.abs(fs - fs0)) <= 1e-14


def test_halfway_differs_from_the_on_node_wall():
    """The flag selects another boundary: the two walls give different states."""
    nx, ny = 24, 10
    runs = []
    for kind in ("wall", "wall_halfway"):
        o = oracle.Oracle(oracle.D2Q4, nx, ny, lam=4.0, omega=1.0, gamma=GAMMA,
                          bc=[("periodic", None)] * 2 + [(kind, None)] * 2)
        runs.append(o.run(o.init(o.prim_to_cons(_fields(nx, ny, 7))), 10)[0])
    assert np.max(np.abs(runs[0] - runs[1])) > 1e-6
