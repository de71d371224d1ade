"""Pins of the oracle's adaptive lattice speed: every collision builds its equilibria with
safety times the largest local bound of the moments before the step and of the Dirichlet
states (the sub-characteristic choice of Section II.C, the bound of Section II.D in 2-D);
every stream advances the time by dx / (the lambda the streamed distributions were built
with); the run stops exactly at a final time.

  AD1  the first chosen lambda (the second step's stream) is safety times the largest bound
       of the initial constant states (Sod: |u| + a of both sides; a four-quadrant problem:
       the D2Q4 bound of its states); the first step streams with the configured lambda
  AD2  at omega = 1 each D1Q2 step is Lax-Friedrichs with its stream lambda
  AD3  the run ends at t_final exactly and the stream time steps sum to it
  AD4  Sod with the adaptive lambda converges to the exact Riemann solution
  AD5  conservation on a periodic grid while lambda changes (omega != 1)
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from workloads import riemann

G = 1.4


def sod_run(n, safety, t_final=0.2):
    wl = W.sod(n)
    o = oracle.Oracle.from_workload(wl)
    fs, lam, t, _ = o.run_adaptive(o.init(o.prim_to_cons(wl.prim)), 100000, wl.dx, safety, t_final)
    return wl, o, fs, lam, t


@pytest.mark.parametrize("safety", [1.0, 1.3])
def test_ad1_first_lambda_sod(safety):
    wl, _, _, lam, _ = sod_run(200, safety)
    a_l, a_r = math.sqrt(G * 1.0 / 1.0), math.sqrt(G * 0.1 / 0.125)
    assert lam[0] == wl.lam
    assert lam[1] == pytest.approx(safety * max(a_l, a_r), rel=1e-15)


def test_ad1_first_lambda_quadrants():
    wl = W.quadrant_riemann(3, 32, steps=0)
    o = oracle.Oracle.from_workload(wl)
    _, lam, _, lam_next = o.run_adaptive(o.init(o.prim_to_cons(wl.prim)), 1, wl.dx, 1.2)
    want = 1.2 * max(W.bouchut_speed(G, *wl.meta["quadrants"][q]) for q in (1, 2, 3, 4))
    assert lam[0] == wl.lam
    assert lam_next == pytest.approx(want, rel=1e-14)


def test_ad2_omega1_is_lax_friedrichs_with_each_lambda():
    wl, o, fs, lam, t = sod_run(120, 1.1, t_final=0.05)
    U = o.prim_to_cons(wl.prim)
    for lam_n in lam:
        rho, m, en = U
        u = m / rho
        p = (G - 1) * (en - 0.5 * m * u)
        F = np.array([m, m * u + p, u * (en + p)])
        Up = np.concatenate([U[:, 1:], U[:, -1:]], 1)
        Um = np.concatenate([U[:, :1], U[:, :-1]], 1)
        Fp = np.concatenate([F[:, 1:], F[:, -1:]], 1)
        Fm = np.concatenate([F[:, :1], F[:, :-1]], 1)
        U = 0.5 * (Up + Um) - (Fp - Fm) / (2 * lam_n)
    assert np.max(np.abs(o.moments(fs) - U)) < 1e-12


@pytest.mark.parametrize("t_final", [0.05, 0.2])
def test_ad3_ends_at_t_final_above_the_bound(t_final):
    wl, o, fs, lam, t = sod_run(300, 1.0, t_final)
    assert t == t_final
    assert np.sum(wl.dx / lam) == pytest.approx(t_final, rel=1e-12)
    # the run stays physical and no lambda falls below the smallest sound speed present
    prim = o.cons_to_prim(o.moments(fs))
    assert prim[0].min() > 0 and prim[2].min() > 0
    assert np.all(lam >= math.sqrt(G * 0.1 / 0.125) - 1e-12)


def test_ad4_sod_converges():
    errs = []
    for n in (250, 500, 1000, 2000):
        wl, o, fs, lam, t = sod_run(n, 1.0)
        ex = riemann.sample(G, wl.meta["left"], wl.meta["right"], (wl.x - 0.5) / 0.2)[0]
        errs.append(np.mean(np.abs(o.moments(fs)[0] - ex)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 0.3) & (orders < 1.0)), errs
    assert errs[2] < 0.0075


@pytest.mark.parametrize("omega", [0.8, 1.6])
def test_ad5_conservation_periodic(omega):
    wl, _ = W.adjoint_pulses(seed=1, n=32, steps=0, width=0.1, pulses=3)
    o = oracle.Oracle(oracle.D2Q4, 32, 32, lam=3.0, omega=omega, bc=wl.bc)
    fs0 = o.init(o.prim_to_cons(wl.prim))
    fs, lam, _, _ = o.run_adaptive(fs0, 80, wl.dx, 1.1)
    assert np.ptp(lam) > 0          # lambda did change
    assert np.allclose(o.moments(fs).sum((1, 2)), o.moments(fs0).sum((1, 2)), rtol=1e-13, atol=1e-13)


def test_ad6_dirichlet_states_count():
    """The oblique-shock problem starts at the inflow state; its top side holds the post-shock
    state, whose bound is the larger: the first chosen lambda must come from it."""
    wl = W.oblique_shock_reflection(nx=64, ny=16, steps=0)
    o = oracle.Oracle.from_workload(wl)
    _, _, _, lam_next = o.run_adaptive(o.init(o.prim_to_cons(wl.prim)), 1, wl.dx, 1.05)
    top = wl.bc[3][1]
    assert W.bouchut_speed(G, *top) > W.bouchut_speed(G, *wl.bc[0][1])
    assert lam_next == pytest.approx(1.05 * W.bouchut_speed(G, *top), rel=1e-14)
