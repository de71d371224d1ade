"""Pins of the oracle's scalar D2Q4 lattice: the 2-D inviscid Burgers law of Section III,
u_t + (u^2/2)_x + u_y = 0, f^eq_q = u/4 + sx g1/(4 lambda) + sy g2/(4 lambda) (Section II.D).

  B1  moment identities: sum_q f^eq = u, lambda sum sx f^eq = u^2/2, lambda sum sy f^eq = u
  B2  at omega = 1 the step is the diagonal four-point scheme on u
  B3  both Section III problems converge to their exact steady solutions (characteristics
      and the shock from the focus), at first order
  B4  conservation of sum u on a periodic grid
  B5  a y-independent state on a y-periodic grid stays y-independent
  B6  brute force on a tiny grid with a linear Dirichlet profile and corner ghosts
  B7  the lambda check reports |u| + 1 (f^eq non-decreasing in u for every population)
"""
import numpy as np
import pytest

import oracle
import workloads as W

P = ("periodic", None)
T = ("transmissive", None)
SX, SY = [-1, 1, 1, -1], [-1, -1, 1, 1]


def burgers(nx, ny, lam, bc, omega=1.0, dx=None):
    return oracle.Oracle(oracle.D2Q4S, nx, ny, lam=lam, omega=omega, bc=bc, dx=dx or 1.0 / nx)


def test_b1_moments():
    rng = np.random.default_rng(0)
    u = rng.uniform(-2, 2, (1, 50))
    lam = 3.7
    o = burgers(50, 1, lam, [P] * 4)
    f = o.feq(u)
    sx, sy = np.array(SX), np.array(SY)
    assert np.allclose(f.sum(0), u, rtol=1e-15, atol=1e-15)
    assert np.allclose(lam * np.tensordot(sx, f, 1), 0.5 * u * u, rtol=1e-13, atol=1e-14)
    assert np.allclose(lam * np.tensordot(sy, f, 1), u, rtol=1e-13, atol=1e-14)


def test_b2_omega1_four_point_scheme():
    n, lam = 24, 3.0
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    u = 0.5 + 0.4 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    o = burgers(n, n, lam, [P] * 4)
    fs, _ = o.run(o.init(u[None]), 30)

    def at(a, di, dj):      # a(i + di, j + dj) on the periodic grid
        return np.roll(np.roll(a, -dj, 0), -di, 1)
    for _ in range(30):
        g1, g2 = 0.5 * u * u, u
        u = (0.25 * (at(u, 1, 1) + at(u, -1, 1) + at(u, -1, -1) + at(u, 1, -1))
             + (-at(g1, 1, 1) - at(g2, 1, 1) + at(g1, -1, 1) - at(g2, -1, 1)
                + at(g1, -1, -1) + at(g2, -1, -1) - at(g1, 1, -1) + at(g2, 1, -1)) / (4 * lam))
    assert np.max(np.abs(o.moments(fs)[0] - u)) < 1e-13


@pytest.mark.parametrize("case", [1, 2])
def test_b3_converges_to_exact_steady_solution(case):
    errs = []
    for n in (32, 64, 128):
        wl = W.burgers_2d(case, n)
        o = oracle.Oracle.from_workload(wl)
        fs, chk = o.run(o.init(wl.prim), wl.steps)
        assert chk["first_bad_step"] == -1
        x = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(x, x)
        errs.append(np.mean(np.abs(o.moments(fs)[0] - W.burgers_steady_exact(case, X, Y))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 0.6) & (orders < 1.3)), (errs, orders)
    assert errs[-1] < (0.03 if case == 1 else 0.045), errs


@pytest.mark.parametrize("omega", [0.8, 1.0, 1.6])
def test_b4_conservation_periodic(omega):
    rng = np.random.default_rng(1)
    n = 32
    u = rng.uniform(-1, 1, (1, n, n))
    o = burgers(n, n, 3.0, [P] * 4, omega)
    fs, _ = o.run(o.init(u), 200)
    assert abs(o.moments(fs).sum() - u.sum()) <= 1e-12 * np.abs(u).sum()


def test_b5_y_independent_state_stays_y_independent():
    n = 40
    x = (np.arange(n) + 0.5) / n
    u = np.broadcast_to(0.3 + 0.5 * np.sin(2 * np.pi * x), (16, n))[None].copy()
    o = burgers(n, 16, 2.5, [T, T, P, P], 1.3)
    fs, _ = o.run(o.init(u), 60)
    U = o.moments(fs)[0]
    assert np.all(U == U[:1])


def test_b6_brute_force_profile_and_corners():
    rng = np.random.default_rng(2)
    nx, ny, lam, dx = 5, 4, 3.0, 0.25
    bc = [("dirichlet", (0.7, 0.3, 0, 0)), T, ("dirichlet", (1.2, -0.8, 0, 0)), ("dirichlet", (-0.4, 0.1, 0, 0))]
    o = burgers(nx, ny, lam, bc, 1.0, dx)
    fs = rng.standard_normal((4, 1, ny, nx))

    def feq(w):
        return [w / 4 + SX[q] * 0.5 * w * w / (4 * lam) + SY[q] * w / (4 * lam) for q in range(4)]

    want = np.empty_like(fs)
    for j in range(ny):
        for i in range(nx):
            for q in range(4):
                si, sj = i - SX[q], j - SY[q]
                if si < 0:                                   # x side first: left profile along y
                    want[q, 0, j, i] = feq(0.7 + 0.3 * (sj + 0.5) * dx)[q]
                    continue
                si = min(si, nx - 1)                         # right side transmissive
                if sj < 0:
                    want[q, 0, j, i] = feq(1.2 - 0.8 * (si + 0.5) * dx)[q]
                elif sj >= ny:
                    want[q, 0, j, i] = feq(-0.4 + 0.1 * (si + 0.5) * dx)[q]
                else:
                    want[q, 0, j, i] = fs[q, 0, sj, si]
    assert np.allclose(o.stream(fs), want, rtol=1e-15, atol=1e-15)


def test_b7_lambda_check():
    u = np.full((1, 6, 6), -1.7)
    o = burgers(6, 6, 3.0, [P] * 4)
    _, chk = o.run(o.init(u), 1)
    assert chk["max_lambda_local"] == pytest.approx(2.7, rel=1e-15)
    o = burgers(6, 6, 2.6, [P] * 4)
    _, chk = o.run(o.init(u), 1)
    assert chk["first_bad_step"] == 1 and chk["n_subchar"] == 36
