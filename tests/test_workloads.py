"""Pins of the exact Riemann solver and the oblique-shock relations, and checks of the generators.

The exact Riemann solver is the reference of the shock-tube convergence pin;
it is pinned here by the conservation laws themselves (Rankine-Hugoniot
jumps across its shocks, isentropy and the Riemann invariant across its fans,
continuity of u and p across its contact).  The oblique-shock state is
pinned by the values the paper prints (tests/golden/oblique_shock_post_state.txt).
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from workloads import riemann
from workloads.oblique import post_shock_state

G = 1.4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def flux1d(rho, u, p):
    E = p / (rho * (G - 1)) + 0.5 * u * u
    return np.array([rho * u, rho * u * u + p, u * (rho * E + p)]), np.array([rho, rho * u, rho * E])


def random_problems(n=40, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        wl = (rng.uniform(0.05, 2), rng.uniform(-1, 1), rng.uniform(0.05, 2))
        wr = (rng.uniform(0.05, 2), rng.uniform(-1, 1), rng.uniform(0.05, 2))
        if not riemann.has_vacuum(G, wl, wr):
            out.append((wl, wr))
    return out


@pytest.mark.parametrize("wl,wr", random_problems())
def test_riemann_waves_satisfy_conservation(wl, wr):
    st = riemann.solve(G, wl, wr)
    sides = [(wl, (st.rho_l, st.u, st.p), st.left_shock, st.sl_head),
             (wr, (st.rho_r, st.u, st.p), st.right_shock, st.sr_head)]
    for w0, ws, is_shock, s in sides:
        if is_shock:
            # Rankine-Hugoniot: F(W*) - F(W0) = S (U(W*) - U(W0))
            F0, U0 = flux1d(*w0)
            F1, U1 = flux1d(*ws)
            assert np.allclose(F1 - F0, s * (U1 - U0), rtol=1e-9, atol=1e-11)
            assert ws[2] > w0[2]  # compressive
        else:
            # isentropic fan: p / rho^gamma constant, Riemann invariant u +/- 2a/(gamma-1) constant
            assert ws[2] / ws[0] ** G == pytest.approx(w0[2] / w0[0] ** G, rel=1e-10)
            a0 = math.sqrt(G * w0[2] / w0[0])
            a1 = math.sqrt(G * ws[2] / ws[0])
            sign = 1.0 if w0 is wl else -1.0
            assert ws[1] + sign * 2 * a1 / (G - 1) == pytest.approx(w0[1] + sign * 2 * a0 / (G - 1), abs=1e-10)


def test_riemann_sampling_is_consistent():
    wl, wr = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    st = riemann.solve(G, wl, wr)
    xi = np.linspace(-3, 3, 2001)
    w = riemann.sample(G, wl, wr, xi)
    assert np.allclose(w[:, 0], wl) and np.allclose(w[:, -1], wr)
    # continuity through the fan, u and p continuous across the contact
    fan = (xi > st.sl_head) & (xi < st.sl_tail)
    assert np.all(np.abs(np.diff(w[0, fan])) < 5e-3)
    near = np.abs(xi - st.u) < 0.01
    assert np.ptp(w[2, near]) < 1e-12 and np.ptp(w[1, near]) < 1e-12
    # Sod: shock at 0.5 + 0.2 S, fan head at 0.5 + 0.2 (u_L - a_L)
    assert 0.5 + 0.2 * st.sl_head == pytest.approx(0.5 - 0.2 * math.sqrt(1.4), rel=1e-12)


def test_vacuum_detected():
    assert riemann.has_vacuum(G, (1.0, -5.0, 0.1), (1.0, 5.0, 0.1))
    with pytest.raises(ValueError):
        riemann.solve(G, (1.0, -5.0, 0.1), (1.0, 5.0, 0.1))


def _golden_oblique():
    vals = {}
    with open(os.path.join(GOLDEN, "oblique_shock_post_state.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, *nums = line.split()
                vals[name] = [float(x) for x in nums]
    return vals


def test_oblique_shock_matches_paper_printed_state():
    g = _golden_oblique()
    rho1, u1, v1, p1 = g["inflow"]
    got = post_shock_state(G, rho1, u1, p1, 29.0)
    # the paper prints 6 significant digits
    assert np.allclose(got, g["post_shock"], rtol=0, atol=1.5e-5), got


def test_oblique_shock_conservation():
    """Normal mass/momentum/energy fluxes continuous across the shock."""
    r1, u1, p1 = 1.0, 2.9, 1 / 1.4
    r2, u2, v2, p2 = post_shock_state(G, r1, u1, p1, 29.0)
    b = math.radians(29.0)
    n = np.array([math.sin(b), math.cos(b)])
    t = np.array([math.cos(b), -math.sin(b)])
    V1, V2 = np.array([u1, 0.0]), np.array([u2, v2])
    vn1, vn2 = V1 @ n, V2 @ n
    assert r1 * vn1 == pytest.approx(r2 * vn2, rel=1e-13)
    assert r1 * vn1 ** 2 + p1 == pytest.approx(r2 * vn2 ** 2 + p2, rel=1e-13)
    h1 = G / (G - 1) * p1 / r1 + 0.5 * vn1 ** 2
    h2 = G / (G - 1) * p2 / r2 + 0.5 * vn2 ** 2
    assert h1 == pytest.approx(h2, rel=1e-13)
    assert V1 @ t == pytest.approx(V2 @ t, rel=1e-13)


def test_generators_are_seeded_and_shaped():
    a = W.quadrant_riemann(3, 32)
    b = W.quadrant_riemann(3, 32)
    assert np.array_equal(a.prim, b.prim) and a.lam == b.lam
    assert a.prim.shape == (4, 32, 32)
    assert not np.array_equal(a.prim, W.quadrant_riemann(4, 32).prim)
    q = a.meta["quadrants"]
    for st in q.values():
        assert 0.1 <= st[0] <= 1.5 and 0.03 <= st[3] <= 1.5 and abs(st[1]) <= 1.2 and abs(st[2]) <= 1.2
    s = W.sod(1000)
    assert s.steps * s.dx / s.lam == pytest.approx(0.2, rel=1e-12)
    tb = W.batched_tubes(0, 64)
    assert tb.lengths.min() >= 200 and tb.lengths.max() <= 20000
    assert np.allclose(tb.steps / (tb.lam * tb.lengths), 0.15, rtol=1e-9)
    assert tb.prim().shape == (3, tb.total_cells)


def test_lambda_bounds_exact_wave_speeds():
    for wl, wr in random_problems(10, seed=3):
        lam = W.lambda_1d_riemann(G, wl, wr, safety=1.0)
        st = riemann.solve(G, wl, wr)
        assert lam >= max(abs(st.sl_head), abs(st.sr_head)) - 1e-12
