"""Exact solution of the 1-D Euler Riemann problem for an ideal gas.

The paper compares its shock-tube results with the analytical solution
(Section III, "Sod's shock tube", citing Toro's textbook).  This module
restates that textbook construction from the gas dynamics:

* the star pressure p* is the root of  f_L(p) + f_R(p) + (u_R - u_L) = 0,
  where f_K is the shock (Rankine-Hugoniot) branch for p > p_K and the
  isentropic rarefaction branch for p <= p_K;
* u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2;
* the star densities follow from the Hugoniot or the isentrope;
* the self-similar solution W(x/t) is sampled wave by wave.

It holds no arithmetic of the lattice Boltzmann relaxation scheme.  It is used
for two things: choosing the lattice speed lambda of a workload from the wave
speeds of its Riemann problems, and as the exact reference of the shock-tube
convergence checks.  Plain numpy/scipy, float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass(frozen=True)
class StarState:
    """Solution of one Riemann problem: star region plus the four wave speeds."""

    p: float           # star pressure
    u: float           # star (contact) velocity
    rho_l: float       # density left of the contact
    rho_r: float       # density right of the contact
    left_shock: bool
    right_shock: bool
    # speeds of the left wave (head, tail) and right wave (tail, head);
    # for a shock head == tail == shock speed
    sl_head: float
    sl_tail: float
    sr_tail: float
    sr_head: float


def sound_speed(gamma: float, rho: float, p: float) -> float:
    return math.sqrt(gamma * p / rho)


def _f_branch(p: float, rho_k: float, p_k: float, a_k: float, gamma: float) -> float:
    """Velocity jump across the K-wave as a function of the star pressure."""
    if p > p_k:  # shock: Rankine-Hugoniot
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        return (p - p_k) * math.sqrt(A / (p + B))
    # rarefaction: isentrope + Riemann invariant
    return 2.0 * a_k / (gamma - 1.0) * ((p / p_k) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def has_vacuum(gamma: float, wl, wr) -> bool:
    """True if the data (rho, u, p) generate vacuum (pressure positivity fails)."""
    rl, ul, pl = wl
    rr, ur, pr = wr
    al, ar = sound_speed(gamma, rl, pl), sound_speed(gamma, rr, pr)
    return 2.0 * (al + ar) / (gamma - 1.0) <= (ur - ul)


def solve(gamma: float, wl, wr) -> StarState:
    """Star state of the Riemann problem with left/right primitive states (rho, u, p)."""
    rl, ul, pl = map(float, wl)
    rr, ur, pr = map(float, wr)
    if min(rl, rr, pl, pr) <= 0.0:
        raise ValueError("Riemann data must have positive density and pressure")
    if has_vacuum(gamma, wl, wr):
        raise ValueError("Riemann data generate vacuum")
    al, ar = sound_speed(gamma, rl, pl), sound_speed(gamma, rr, pr)
    du = ur - ul

    def phi(p):
        return _f_branch(p, rl, pl, al, gamma) + _f_branch(p, rr, pr, ar, gamma) + du

    lo, hi = 1e-14 * min(pl, pr), 10.0 * max(pl, pr)
    while phi(hi) < 0.0:
        hi *= 10.0
    ps = brentq(phi, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_f_branch(ps, rr, pr, ar, gamma) - _f_branch(ps, rl, pl, al, gamma))

    g1 = (gamma - 1.0) / (gamma + 1.0)
    # left wave
    if ps > pl:
        rho_l = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
        s = ul - al * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + (gamma - 1.0) / (2.0 * gamma))
        sl_head = sl_tail = s
        lshock = True
    else:
        rho_l = rl * (ps / pl) ** (1.0 / gamma)
        a_star = al * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
        sl_head, sl_tail = ul - al, us - a_star
        lshock = False
    # right wave
    if ps > pr:
        rho_r = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
        s = ur + ar * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
        sr_head = sr_tail = s
        rshock = True
    else:
        rho_r = rr * (ps / pr) ** (1.0 / gamma)
        a_star = ar * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
        sr_tail, sr_head = us + a_star, ur + ar
        rshock = False
    return StarState(ps, us, rho_l, rho_r, lshock, rshock, sl_head, sl_tail, sr_tail, sr_head)


def sample(gamma: float, wl, wr, xi) -> np.ndarray:
    """Exact solution (rho, u, p) at similarity coordinates xi = (x - x0)/t.

    Returns an array of shape (3, len(xi)).
    """
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    rl, ul, pl = map(float, wl)
    rr, ur, pr = map(float, wr)
    st = solve(gamma, wl, wr)
    al, ar = sound_speed(gamma, rl, pl), sound_speed(gamma, rr, pr)
    out = np.empty((3, xi.size))
    gm1, gp1 = gamma - 1.0, gamma + 1.0
    for n, s in enumerate(xi):
        if s <= st.u:  # left of the contact
            if s <= st.sl_head:
                w = (rl, ul, pl)
            elif s >= st.sl_tail:
                w = (st.rho_l, st.u, st.p)
            else:  # inside the left fan
                u = 2.0 / gp1 * (al + 0.5 * gm1 * ul + s)
                a = 2.0 / gp1 * (al + 0.5 * gm1 * (ul - s))
                w = (rl * (a / al) ** (2.0 / gm1), u, pl * (a / al) ** (2.0 * gamma / gm1))
        else:
            if s >= st.sr_head:
                w = (rr, ur, pr)
            elif s <= st.sr_tail:
                w = (st.rho_r, st.u, st.p)
            else:  # inside the right fan
                u = 2.0 / gp1 * (-ar + 0.5 * gm1 * ur + s)
                a = 2.0 / gp1 * (ar - 0.5 * gm1 * (ur - s))
                w = (rr * (a / ar) ** (2.0 / gm1), u, pr * (a / ar) ** (2.0 * gamma / gm1))
        out[:, n] = w
    return out


def star_states(gamma: float, wl, wr):
    """The constant states of the solution, left to right: W_L, W*_L, W*_R, W_R.

    Inside a rarefaction fan the extreme values of |u|, |u -/+ a| and the
    diagonal speeds used below are reached at the fan's edges, so these four
    states bound every wave speed of the exact solution.
    """
    st = solve(gamma, wl, wr)
    return [tuple(map(float, wl)), (st.rho_l, st.u, st.p), (st.rho_r, st.u, st.p), tuple(map(float, wr))]
