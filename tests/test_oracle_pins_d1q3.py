"""Pins of the oracle's D1Q3 model (rest particle added, Section II.C).

f^eq = (U/3 - G/(2 lambda), U/3, U/3 + G/(2 lambda)) for velocities (-lambda, 0, +lambda).
  Q1  moment identities: sum_q f^eq = U, sum_q lambda_q f^eq = G, rest part U/3
  Q2  at omega = 1 the step is the three-point scheme
      U_j <- (U_{j+1} + U_j + U_{j-1})/3 - (G_{j+1} - G_{j-1})/(2 lambda)
  Q3  uniform flow preserved; conservation on a periodic line
  Q4  steady contact keeps u = 0 and p = 1 exactly
  Q5  Sod converges to the exact Riemann solution, with smaller error than D1Q2
      (the paper: the rest particle removes the D1Q2 staircase)
  Q6  Chapman-Enskog rate dt (1/omega - 1/2)(2 lambda^2/3 - c^2) k^2
      (second moment sum_q lambda_q^2 f^eq = 2 lambda^2 U / 3)
  Q7  the paper's steady Mach-2 shock (run there with this model) stays put
  Q8  brute force on a tiny grid
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from workloads import riemann

G = 1.4


def d1q3(n, lam, omega=1.0, bc="periodic", state=None):
    return oracle.Oracle(oracle.D1Q3, n, lam=lam, omega=omega,
                         bc=[(bc, state if bc == "dirichlet" else None)] * 2)


def flux(U, g=G):
    rho, m, en = U
    u = m / rho
    p = (g - 1) * (en - 0.5 * rho * u * u)
    return np.array([m, m * u + p, u * (en + p)])


def test_q1_moments():
    rng = np.random.default_rng(0)
    n = 200
    prim = np.array([rng.uniform(0.2, 2, n), rng.uniform(-1, 1, n), rng.uniform(0.2, 2, n)])
    lam = 3.3
    o = d1q3(n, lam)
    U = o.prim_to_cons(prim)
    feq = o.feq(U)
    assert feq.shape == (3, 3, n)
    assert np.allclose(feq.sum(0), U, rtol=1e-14, atol=1e-14)
    assert np.allclose(lam * (feq[2] - feq[0]), flux(U), rtol=1e-13, atol=1e-13)
    assert np.allclose(feq[1], U / 3, rtol=1e-15)
    assert np.allclose(lam * lam * (feq[0] + feq[2]), 2 * lam * lam * U / 3, rtol=1e-13)


@pytest.mark.parametrize("bc", ["periodic", "transmissive"])
def test_q2_omega1_three_point_scheme(bc):
    n, lam = 64, 3.0
    x = (np.arange(n) + 0.5) / n
    prim = np.array([1 + 0.3 * np.sin(2 * np.pi * x), 0.2 + 0.3 * np.cos(2 * np.pi * x), 1 + 0.2 * np.sin(4 * np.pi * x)])
    o = d1q3(n, lam, bc=bc)
    U = o.prim_to_cons(prim)
    fs, _ = o.run(o.init(U), 50)
    for _ in range(50):
        F = flux(U)
        if bc == "periodic":
            Up, Um, Fp, Fm = np.roll(U, -1, 1), np.roll(U, 1, 1), np.roll(F, -1, 1), np.roll(F, 1, 1)
        else:
            Up = np.concatenate([U[:, 1:], U[:, -1:]], 1)
            Um = np.concatenate([U[:, :1], U[:, :-1]], 1)
            Fp = np.concatenate([F[:, 1:], F[:, -1:]], 1)
            Fm = np.concatenate([F[:, :1], F[:, :-1]], 1)
        U = (Up + U + Um) / 3 - (Fp - Fm) / (2 * lam)
    assert np.max(np.abs(o.moments(fs) - U)) < 1e-13


@pytest.mark.parametrize("omega", [0.8, 1.0, 1.6])
def test_q3_uniform_and_conservation(omega):
    n = 40
    o = d1q3(n, 3.0, omega)
    prim = np.array([np.full(n, 0.8), np.full(n, 0.3), np.full(n, 1.2)])
    U0 = o.prim_to_cons(prim)
    fs, _ = o.run(o.init(U0), 400)
    assert np.max(np.abs(o.moments(fs) - U0)) <= 1e-14 * np.abs(U0).max()
    x = (np.arange(n) + 0.5) / n
    prim = np.array([1 + 0.2 * np.sin(2 * np.pi * x), 0.1 + 0.2 * np.cos(2 * np.pi * x), 1 + 0.1 * np.sin(6 * np.pi * x)])
    U0 = o.prim_to_cons(prim)
    fs, _ = o.run(o.init(U0), 400)
    assert np.allclose(o.moments(fs).sum(1), U0.sum(1), rtol=1e-13)


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.5])
def test_q4_steady_contact(omega):
    s = W.steady_contact(omega=omega, lattice="d1q3")
    o = oracle.Oracle.from_workload(s, lattice=oracle.D1Q3)
    fs, _ = o.run(o.init(o.prim_to_cons(s.prim)), s.steps)
    prim = o.cons_to_prim(o.moments(fs))
    assert np.max(np.abs(prim[1])) < 1e-14
    assert np.max(np.abs(prim[2] - 1.0)) < 1e-13


def sod_l1(n, lattice):
    s = W.sod(n, lattice="d1q3" if lattice == oracle.D1Q3 else "d1q2")
    o = oracle.Oracle.from_workload(s, lattice=lattice)
    fs, chk = o.run(o.init(o.prim_to_cons(s.prim)), s.steps)
    assert chk["first_bad_step"] == -1
    ex = riemann.sample(G, s.meta["left"], s.meta["right"], (s.x - 0.5) / s.t_final)[0]
    rho = o.moments(fs)[0]
    return np.mean(np.abs(rho - ex)), rho


def test_q5_sod_converges_and_beats_d1q2():
    errs = [sod_l1(n, oracle.D1Q3)[0] for n in (250, 500, 1000, 2000)]
    assert np.all(np.diff(errs) < 0)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 0.3) & (orders < 1.0))
    e3, rho3 = sod_l1(1000, oracle.D1Q3)
    e2, rho2 = sod_l1(1000, oracle.D1Q2)
    assert e3 < e2
    # the D1Q2 staircase (Section III): at omega = 1 the even and odd cells of D1Q2 never
    # exchange data, so the rarefaction fan is a staircase of cell pairs -- its first
    # differences alternate between ~0 and twice the slope.  The rest particle couples
    # the sublattices and the fan is smooth.
    x = W.sod(1000).x
    fan = ((x > 0.28) & (x < 0.47))[:-1]

    def alternation(rho):
        d = np.diff(rho)[fan]
        return np.sum(np.abs(np.diff(d))) / np.sum(np.abs(d))

    assert alternation(rho2) > 1.0
    assert alternation(rho3) < 0.05


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.5])
def test_q6_chapman_enskog_decay(omega):
    n, lam, eps = 64, 2.0, 1e-6
    dx = 1.0 / n
    dt = dx / lam
    k = 2 * np.pi
    x = (np.arange(n) + 0.5) * dx
    a = math.sqrt(G)
    cases = {"entropy": (np.array([1 + eps * np.sin(k * x), 0 * x, 1 + 0 * x]), 0.0, 0),
             "acoustic": (np.array([1 + eps * np.sin(k * x), eps * a * np.sin(k * x), 1 + eps * a * a * np.sin(k * x)]),
                          a, 2)}
    for name, (prim, c, comp) in cases.items():
        o = d1q3(n, lam, omega)
        fs1, _ = o.run(o.init(o.prim_to_cons(prim)), 20)
        fs2, _ = o.run(fs1, 400)

        def amp(fs):
            f = o.cons_to_prim(o.moments(fs))[comp]
            return np.abs(np.fft.rfft(f - f.mean())[1])

        rate = math.log(amp(fs1) / amp(fs2)) / (400 * dt)
        nu = dt * (1 / omega - 0.5) * (2 * lam * lam / 3 - c * c)
        assert rate == pytest.approx(nu * k * k, rel=0.05), (name, rate, nu * k * k)


def test_q7_steady_mach2_shock():
    s = W.steady_shock(nx=400, steps=1000, lattice="d1q3")
    o = oracle.Oracle.from_workload(s, lattice=oracle.D1Q3)
    fs, chk = o.run(o.init(o.prim_to_cons(s.prim)), s.steps)
    rho = o.moments(fs)[0]
    r1, r2 = s.meta["pre"][0], s.meta["post"][0]

    def centroid(r):
        return s.x0 + (np.sum(r2 - r) / (r2 - r1)) * s.dx

    assert chk["first_bad_step"] == -1
    assert abs(centroid(rho) - centroid(s.prim[0])) <= 2 * s.dx


def test_q8_brute_force():
    rng = np.random.default_rng(9)
    n, lam, om = 5, 4.0, 0.8
    prim = np.array([rng.uniform(0.5, 2, n), rng.uniform(-1, 1, n), rng.uniform(0.5, 2, n)])
    o = d1q3(n, lam, om, bc="transmissive")
    fs = o.init(o.prim_to_cons(prim))
    ref = fs.copy()
    for _ in range(2):
        f = np.stack([np.concatenate([ref[0][:, 1:], ref[0][:, -1:]], 1), ref[1],
                      np.concatenate([ref[2][:, :1], ref[2][:, :-1]], 1)])
        U = f.sum(0)
        F = flux(U)
        feq = np.stack([U / 3 - F / (2 * lam), U / 3, U / 3 + F / (2 * lam)])
        ref = (1 - om) * f + om * feq
    got, _ = o.run(fs, 2)
    assert np.max(np.abs(got - ref)) < 1e-14 * np.abs(ref).max()


def test_q9_lattice_speed_bound():
    """The check reports sqrt(3/2)(|u| + a): the speed at which the D1Q3 diffusion
    dt (1/omega - 1/2)(2 lambda^2/3 - c^2) of the fastest wave (c = |u| + a) vanishes."""
    n, state = 8, (0.9, -0.4, 1.3)
    o = d1q3(n, 5.0)
    prim = np.array([np.full(n, s) for s in state])
    _, chk = o.run(o.init(o.prim_to_cons(prim)), 1)
    c = abs(state[1]) + math.sqrt(G * state[2] / state[0])
    assert chk["max_lambda_local"] == pytest.approx(math.sqrt(1.5) * c, rel=1e-14)
    # and a lambda between c and sqrt(3/2) c is flagged
    o = d1q3(n, 1.1 * c)
    _, chk = o.run(o.init(o.prim_to_cons(prim)), 1)
    assert chk["first_bad_step"] == 1 and chk["n_subchar"] == n
