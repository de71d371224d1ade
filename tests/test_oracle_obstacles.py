"""Pins of the oracle's internal walls (lattice-aligned obstacles; Section II.E's free-slip
wall extended to solid cells, Section III's step problems).

  W1  a fluid at rest stays exactly at rest around any obstacles (every reflection maps the
      rest equilibrium onto itself only with the right signs); solid cells are inert
  W2  a solid band along the top (bottom) reproduces the paper's top (bottom) wall row rule
      on the shorter grid, bit for bit
  W3  a solid band along the right (left) side is the transpose of the top (bottom) band run
      (x <-> y, u <-> v, f2 <-> f4): pins the rule for walls normal to x
  W4  a square obstacle in a periodic box keeps the x-mirror, y-mirror and diagonal symmetries
      of a symmetric initial state (corners included)
  W5  brute force on a tiny grid: streaming with an obstacle against a direct restatement
  W6  the paper's forward-facing step (240 x 80, t = 4) and shock diffraction run without
      non-physical cells or lambda violations
  W7  a fluid channel one cell wide is rejected
"""
import numpy as np
import pytest

import oracle
import workloads as W

G = 1.4
SX = [-1, 1, 1, -1]
SY = [-1, -1, 1, 1]


def make(nx, ny, lam, bc, solid, omega=1.0):
    return oracle.Oracle(oracle.D2Q4, nx, ny, lam=lam, omega=omega, bc=bc, solid=solid)


def rects(ny, nx, boxes):
    m = np.zeros((ny, nx), np.uint8)
    for (i0, i1, j0, j1) in boxes:
        m[j0:j1, i0:i1] = 1
    return m


def smooth_state(nx, ny, seed=0):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    a = rng.uniform(0.05, 0.15, 4)
    return np.array([1 + a[0] * np.sin(2 * np.pi * X + 1) * np.cos(2 * np.pi * Y),
                     0.3 + a[1] * np.cos(2 * np.pi * Y + 0.5),
                     -0.2 + a[2] * np.sin(2 * np.pi * X),
                     1 + a[3] * np.cos(2 * np.pi * (X + Y))])


P = ("periodic", None)
T = ("transmissive", None)
WALL = ("wall", None)


@pytest.mark.parametrize("bc", [[P, P, WALL, WALL], [T, T, T, T], [P, P, P, P]])
@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_w1_rest_state_is_kept(bc, omega):
    nx, ny = 40, 30
    solid = rects(ny, nx, [(5, 12, 4, 9), (20, 22, 10, 25), (28, 36, 2, 4), (30, 34, 20, 26)])
    o = make(nx, ny, 3.0, bc, solid, omega)
    prim = np.array([np.full((ny, nx), 1.3), np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), 0.9)])
    U0 = o.prim_to_cons(prim)
    fs0 = o.init(U0)
    fs, chk = o.run(fs0, 60)
    assert chk["first_bad_step"] == -1
    U = o.moments(fs)
    assert np.max(np.abs(U - U0)) <= 1e-13
    # solid cells carry their distributions unchanged
    assert np.array_equal(fs[:, :, solid == 1], fs0[:, :, solid == 1])


@pytest.mark.parametrize("side", ["top", "bottom"])
@pytest.mark.parametrize("xbc", [P, T])
@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_w2_band_equals_paper_wall(side, xbc, omega):
    nx, ny, k = 36, 20, 3
    prim = smooth_state(nx, ny)
    prim[2, -1 if side == "top" else 0, :] = 0.0
    # reference: the paper's wall row on the domain side
    bc_ref = [xbc, xbc, WALL if side == "bottom" else T, WALL if side == "top" else T]
    ref = make(nx, ny, 3.0, bc_ref, None, omega)
    fr, _ = ref.run(ref.init(ref.prim_to_cons(prim)), 40)
    # the same grid grown by k solid rows on that side
    big = np.empty((4, ny + k, nx))
    solid = np.zeros((ny + k, nx), np.uint8)
    if side == "top":
        big[:, :ny] = prim
        big[:, ny:] = prim[:, -1:]
        solid[ny:] = 1
        rows = slice(0, ny)
    else:
        big[:, k:] = prim
        big[:, :k] = prim[:, :1]
        solid[:k] = 1
        rows = slice(k, ny + k)
    o = make(nx, ny + k, 3.0, [xbc, xbc, T, T], solid, omega)
    fb, _ = o.run(o.init(o.prim_to_cons(big)), 40)
    assert np.array_equal(fb[:, :, rows, :], fr)


def transpose_dists(fs):
    """(x, y) -> (y, x): populations (sx, sy) -> (sy, sx), i.e. f1, f3 stay, f2 <-> f4;
    fields rho u <-> rho v."""
    out = fs[[0, 3, 2, 1]][:, [0, 2, 1, 3]]
    return np.ascontiguousarray(np.swapaxes(out, 2, 3))


@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_w3_vertical_band_is_transposed_horizontal_band(side, omega):
    nx, ny, k = 24, 30, 3         # the band problem; its transpose is ny x nx
    prim = smooth_state(nx, ny, seed=1)
    solid = np.zeros((ny, nx), np.uint8)
    if side == "right":
        solid[:, nx - k:] = 1
    else:
        solid[:, :k] = 1
    o = make(nx, ny, 3.0, [T, T, P, P], solid, omega)
    fs, _ = o.run(o.init(o.prim_to_cons(prim)), 30)
    primT = np.ascontiguousarray(np.swapaxes(prim[[0, 2, 1, 3]], 1, 2))
    oT = make(ny, nx, 3.0, [P, P, T, T], np.ascontiguousarray(solid.T), omega)
    fT, _ = oT.run(oT.init(oT.prim_to_cons(primT)), 30)
    fluid = np.swapaxes(solid, 0, 1) == 0
    a, b = transpose_dists(fs)[:, :, fluid], fT[:, :, fluid]
    # the transposed run evaluates the same sums in another order: rounding only
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_w4_square_obstacle_keeps_symmetries(omega):
    n = 32
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    # symmetric under x -> 1 - x, y -> 1 - y and x <-> y (u, v odd / swapped accordingly)
    r = np.hypot(X - 0.5, Y - 0.5)
    prim = np.array([1 + 0.2 * np.exp(-40 * r ** 2), 0.3 * np.sin(2 * np.pi * X) * np.cos(np.pi * (Y - 0.5)) ** 2,
                     0.3 * np.sin(2 * np.pi * Y) * np.cos(np.pi * (X - 0.5)) ** 2, 1 + 0.3 * np.exp(-40 * r ** 2)])
    solid = rects(n, n, [(12, 20, 12, 20)])
    o = make(n, n, 3.0, [P] * 4, solid, omega)
    fs, chk = o.run(o.init(o.prim_to_cons(prim)), 50)
    assert chk["first_bad_step"] == -1
    U = o.moments(fs)
    scale = np.max(np.abs(U))
    # x-mirror: rho, v, E even, rho u odd
    assert np.max(np.abs(U[[0, 2, 3]] - U[[0, 2, 3]][:, :, ::-1])) <= 1e-12 * scale
    assert np.max(np.abs(U[1] + U[1][:, ::-1])) <= 1e-12 * scale
    # y-mirror
    assert np.max(np.abs(U[[0, 1, 3]] - U[[0, 1, 3]][:, ::-1, :])) <= 1e-12 * scale
    assert np.max(np.abs(U[2] + U[2][::-1, :])) <= 1e-12 * scale
    # diagonal: rho, E symmetric, rho u <-> rho v
    assert np.max(np.abs(U[[0, 3]] - np.swapaxes(U[[0, 3]], 1, 2))) <= 1e-12 * scale
    assert np.max(np.abs(U[1] - U[2].T)) <= 1e-12 * scale


def brute_stream(fs, solid):
    """Periodic D2Q4 streaming with the internal-wall rule, restated cell by cell."""
    _, _, ny, nx = fs.shape
    f = np.empty_like(fs)
    for j in range(ny):
        for i in range(nx):
            if solid[j, i]:
                f[:, :, j, i] = fs[:, :, j, i]
                continue
            unknown = []
            for q in range(4):
                si, sj = (i - SX[q]) % nx, (j - SY[q]) % ny
                if solid[sj, si]:
                    unknown.append(q)
                else:
                    f[q, :, j, i] = fs[q, :, sj, si]
            for q in unknown:
                xn = solid[j, (i - SX[q]) % nx]
                yn = solid[(j - SY[q]) % ny, i]
                mx, my = SX[q], SY[q]
                if xn and not yn:
                    mx = -mx
                elif yn and not xn:
                    my = -my
                else:
                    mx, my = -mx, -my
                m = [(a, b) for a, b in zip(SX, SY)].index((mx, my))
                sign = np.array([1.0, -1.0 if mx != SX[q] else 1.0, -1.0 if my != SY[q] else 1.0, 1.0])
                f[q, :, j, i] = sign * f[m, :, j, i]
    return f


def test_w5_brute_force_stream():
    rng = np.random.default_rng(4)
    nx, ny = 9, 8
    solid = rects(ny, nx, [(3, 5, 2, 5), (7, 8, 6, 8)])
    o = make(nx, ny, 4.0, [P] * 4, solid)
    fs = rng.standard_normal((4, 4, ny, nx))
    assert np.array_equal(o.stream(fs), brute_stream(fs, solid))


def test_w6_paper_step_problems_stay_physical():
    for wl in (W.forward_facing_step(), W.shock_diffraction(n=400)):
        o = oracle.Oracle.from_workload(wl)
        fs, chk = o.run(o.init(o.prim_to_cons(wl.prim)), wl.steps)
        assert chk["first_bad_step"] == -1, (wl.name, chk)
        assert chk["max_lambda_local"] < wl.lam
        prim = o.cons_to_prim(o.moments(fs))
        fluid = wl.solid == 0
        assert prim[0][fluid].min() > 0 and prim[3][fluid].min() > 0


def test_w7_one_cell_channel_rejected():
    solid = rects(10, 12, [(0, 12, 0, 4), (0, 12, 5, 10)])
    with pytest.raises(ValueError, match="mirror"):
        make(12, 10, 3.0, [P] * 4, solid)
