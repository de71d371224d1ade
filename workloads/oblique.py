"""Oblique-shock relations of an ideal gas.

The oblique shock reflection case of the paper (Section III, "Oblique shock
reflection test case") holds the top boundary at the state behind an oblique
shock, "calculated from the oblique shock relations from gas dynamics".  This
module restates those relations: the velocity component normal to the shock
jumps by the normal-shock (Rankine-Hugoniot) relations at the normal Mach
number M sin(beta); the tangential component is unchanged.

No lattice Boltzmann arithmetic lives here.
"""
from __future__ import annotations

import math


def post_shock_state(gamma: float, rho1: float, u1: float, p1: float, beta_deg: float):
    """State (rho, u, v, p) behind a shock inclined at beta to a uniform flow (rho1, u1, 0, p1).

    The shock runs down and to the right (it enters through the top-left of a
    channel), so the flow behind it is turned towards the lower wall (v < 0).
    """
    beta = math.radians(beta_deg)
    a1 = math.sqrt(gamma * p1 / rho1)
    mn1 = u1 * math.sin(beta) / a1
    if mn1 <= 1.0:
        raise ValueError("normal Mach number must exceed 1 for a shock")
    rho2 = rho1 * (gamma + 1.0) * mn1 * mn1 / ((gamma - 1.0) * mn1 * mn1 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (mn1 * mn1 - 1.0))
    vt = u1 * math.cos(beta)             # tangential component, continuous
    vn2 = u1 * math.sin(beta) * rho1 / rho2  # normal component, from mass flux
    # tangent t = (cos b, -sin b), normal n = (sin b, cos b)
    u2 = vt * math.cos(beta) + vn2 * math.sin(beta)
    v2 = -vt * math.sin(beta) + vn2 * math.cos(beta)
    return rho2, u2, v2, p2
