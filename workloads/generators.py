"""Workload builders: the paper's test problems and their seeded synthetic stand-ins.

Conventions shared by every consumer:

* cells are cell-centred, x_i = x0 + (i + 1/2) dx (and likewise in y);
* 2-D primitive fields have shape (4, ny, nx) in the order (rho, u, v, p),
  1-D fields shape (3, nx) in the order (rho, u, p);
* boundary conditions are given per side (x-lo, x-hi[, y-lo, y-hi]) as
  ``(kind, state)`` with kind one of "periodic", "transmissive", "dirichlet",
  "wall" and state the primitive Dirichlet state (or None);
* lambda is one global lattice speed for the whole run (exact hopping needs a
  single dt = dx / lambda, Eq. for the discrete LBRS update, Section II.A).

Lambda is chosen from the exact Riemann solutions of the initial
discontinuities: the largest local speed over every constant state of those
solutions (the 1-D formula max(|u-a|, |u|, |u+a|) of Section II.C, or the
Bouchut bound of Section II.D for D2Q4, read as max(|u+v|, |u-v|) + sqrt(2) a),
times a safety factor.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import riemann
from .oblique import post_shock_state

GAMMA = 1.4


@dataclass
class Workload1D:
    name: str
    nx: int
    dx: float
    x0: float
    prim: np.ndarray            # (3, nx) rho, u, p
    bc: list                    # [(kind, state_or_None)] * 2
    lam: float
    omega: float
    steps: int
    gamma: float = GAMMA
    t_final: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def x(self) -> np.ndarray:
        return self.x0 + (np.arange(self.nx) + 0.5) * self.dx


@dataclass
class Workload2D:
    name: str
    nx: int
    ny: int
    dx: float
    x0: float
    y0: float
    prim: np.ndarray            # (4, ny, nx) rho, u, v, p
    bc: list                    # [(kind, state_or_None)] * 4: x-lo, x-hi, y-lo, y-hi
    lam: float
    omega: float
    steps: int
    gamma: float = GAMMA
    meta: dict = field(default_factory=dict)
    solid: np.ndarray | None = None   # (ny, nx) uint8, 1 = solid cell of an internal wall
    law: str = "euler"                 # "euler" (4 fields) or "burgers" (the scalar law, 1 field)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


@dataclass
class TubeBatch:
    """Many independent 1-D shock tubes of uneven length, each on [0, 1]."""

    lengths: np.ndarray         # (B,) int64 cells per tube
    left: np.ndarray            # (B, 3) rho, u, p left of x = 0.5
    right: np.ndarray           # (B, 3)
    lam: np.ndarray             # (B,) lattice speed per tube
    steps: np.ndarray           # (B,) steps per tube to reach t_final
    t_final: float
    omega: float
    gamma: float = GAMMA
    lattice: str = "d1q2"       # "d1q2" or "d1q3" (lambda scaled by LAMBDA_FACTOR)

    @property
    def total_cells(self) -> int:
        return int(self.lengths.sum())

    @property
    def total_updates(self) -> int:
        return int((self.lengths * self.steps).sum())

    def subset(self, idx) -> "TubeBatch":
        """The tubes idx (in that order) as a batch of their own."""
        idx = np.asarray(idx, dtype=np.int64)
        return TubeBatch(self.lengths[idx], self.left[idx], self.right[idx], self.lam[idx], self.steps[idx],
                         self.t_final, self.omega, self.gamma, self.lattice)

    def prim(self) -> np.ndarray:
        """Concatenated primitive fields, shape (3, sum N), tube b at offset sum_{c<b} N_c."""
        out = np.empty((3, self.total_cells))
        off = 0
        for b, n in enumerate(self.lengths):
            n = int(n)
            xc = (np.arange(n) + 0.5) / n
            for k in range(3):
                out[k, off:off + n] = np.where(xc < 0.5, self.left[b, k], self.right[b, k])
            off += n
        return out


def sound(gamma, rho, p):
    return math.sqrt(gamma * p / rho)


def bouchut_speed(gamma, rho, u, v, p) -> float:
    """Largest of |u+v|, |u-v| plus sqrt(2) a: the D2Q4 Euler bound of Section II.D."""
    return max(abs(u + v), abs(u - v)) + math.sqrt(2.0) * sound(gamma, rho, p)


def _round_lambda(lam: float, dx: float, t_final: float):
    """Raise lambda so that t_final / dt = t_final * lambda / dx is an integer."""
    n = int(math.ceil(t_final * lam / dx - 1e-9))
    return n * dx / t_final, n


def lambda_1d_riemann(gamma, wl, wr, safety=1.05, lam_min=0.0) -> float:
    """max(|u|+a) over the constant states of the exact solution, times safety."""
    states = riemann.star_states(gamma, wl, wr)
    lam = max(abs(u) + sound(gamma, r, p) for (r, u, p) in states)
    return max(lam_min, safety * lam)


def lambda_2d_quadrants(gamma, q, safety=1.1) -> float:
    """Bouchut bound over the four interface Riemann problems of a quadrant problem.

    q maps 1..4 (quadrants counter-clockwise from the top right) to (rho, u, v, p).
    Across an x-interface u is normal and v is carried by each side; across a
    y-interface v is normal and u is carried.
    """
    lam = 0.0
    # x-interfaces: (left, right) = (2, 1) on top, (3, 4) at the bottom
    for a, b in ((2, 1), (3, 4)):
        (ra, ua, va, pa), (rb, ub, vb, pb) = q[a], q[b]
        sts = riemann.star_states(gamma, (ra, ua, pa), (rb, ub, pb))
        tang = (va, va, vb, vb)
        for (r, un, p), vt in zip(sts, tang):
            lam = max(lam, bouchut_speed(gamma, r, un, vt, p))
    # y-interfaces: (lower, upper) = (4, 1) right, (3, 2) left
    for a, b in ((4, 1), (3, 2)):
        (ra, ua, va, pa), (rb, ub, vb, pb) = q[a], q[b]
        sts = riemann.star_states(gamma, (ra, va, pa), (rb, vb, pb))
        tang = (ua, ua, ub, ub)
        for (r, vn, p), ut in zip(sts, tang):
            lam = max(lam, bouchut_speed(gamma, r, ut, vn, p))
    return safety * lam


# --------------------------------------------------------------------------- 1-D

# D1Q3 carries (2/3) lambda^2 U in its second moment, so its lattice speed must
# exceed sqrt(3/2) times the wave speeds (positive Chapman-Enskog diffusion).
LAMBDA_FACTOR = {"d1q2": 1.0, "d1q3": math.sqrt(1.5)}


def sod(nx: int = 1000, omega: float = 1.0, t_final: float = 0.2, lattice: str = "d1q2") -> Workload1D:
    """Sod's shock tube in nondimensional form on [0, 1], diaphragm at 0.5 (Section III).

    The paper runs the dimensional version (1 kg/m^3, 0, 1e5 Pa | 0.125, 0,
    1e4 Pa) on [-10, 10]; this is the usual scaled form with the same ratios.
    """
    wl, wr = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    dx = 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    prim = np.empty((3, nx))
    for k in range(3):
        prim[k] = np.where(x < 0.5, wl[k], wr[k])
    lam, steps = _round_lambda(LAMBDA_FACTOR[lattice] * lambda_1d_riemann(GAMMA, wl, wr), dx, t_final)
    return Workload1D("sod", nx, dx, 0.0, prim, [("transmissive", None)] * 2, lam, omega, steps,
                      t_final=t_final, meta={"left": wl, "right": wr, "x_interface": 0.5})


def steady_contact(nx: int = 100, omega: float = 1.0, t_final: float = 2.0, lattice: str = "d1q2") -> Workload1D:
    """Stationary contact (rho 1.4 | 1.0, u = 0, p = 1) on [0, 1] (Section III)."""
    wl, wr = (1.4, 0.0, 1.0), (1.0, 0.0, 1.0)
    dx = 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    prim = np.empty((3, nx))
    for k in range(3):
        prim[k] = np.where(x < 0.5, wl[k], wr[k])
    lam0 = 1.05 * LAMBDA_FACTOR[lattice] * max(sound(GAMMA, 1.0, 1.0), sound(GAMMA, 1.4, 1.0))
    lam, steps = _round_lambda(lam0, dx, t_final)
    return Workload1D("steady_contact", nx, dx, 0.0, prim, [("transmissive", None)] * 2, lam, omega,
                      steps, t_final=t_final, meta={"left": wl, "right": wr})


def steady_shock(nx: int = 400, mach: float = 2.0, omega: float = 1.0, steps: int = 1000,
                 lattice: str = "d1q2") -> Workload1D:
    """Stationary Mach-2 normal shock at x = 0 on [-1, 1] (Section III, steady shock).

    Pre-shock state (1, M a, 1/gamma) so that a = 1; the post-shock state
    comes from the normal-shock relations.
    """
    r1, p1 = 1.0, 1.0 / GAMMA
    u1 = mach * sound(GAMMA, r1, p1)
    r2 = r1 * (GAMMA + 1) * mach ** 2 / ((GAMMA - 1) * mach ** 2 + 2)
    p2 = p1 * (1 + 2 * GAMMA / (GAMMA + 1) * (mach ** 2 - 1))
    u2 = u1 * r1 / r2
    dx = 2.0 / nx
    x = -1.0 + (np.arange(nx) + 0.5) * dx
    prim = np.empty((3, nx))
    for k, (a, b) in enumerate(zip((r1, u1, p1), (r2, u2, p2))):
        prim[k] = np.where(x < 0.0, a, b)
    lam = 1.1 * LAMBDA_FACTOR[lattice] * max(abs(u1) + sound(GAMMA, r1, p1), abs(u2) + sound(GAMMA, r2, p2))
    bc = [("dirichlet", (r1, u1, p1)), ("dirichlet", (r2, u2, p2))]
    return Workload1D("steady_shock", nx, dx, -1.0, prim, bc, lam, omega, steps,
                      meta={"pre": (r1, u1, p1), "post": (r2, u2, p2)})


def batched_tubes(seed: int = 0, count: int = 4096, n_min: int = 200, n_max: int = 20000,
                  t_final: float = 0.15, omega: float = 1.0, lattice: str = "d1q2") -> TubeBatch:
    """Seeded shock tubes on [0, 1] with log-uniform lengths.

    Left/right rho, p ~ U[0.05, 2], u ~ U[-1, 1]; a draw whose Riemann problem
    generates vacuum is replaced by the next draw.  Lambda per tube from its
    exact solution (times the lattice's factor), rounded so t_final is reached in
    a whole number of steps.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count))).astype(np.int64)
    left = np.empty((count, 3))
    right = np.empty((count, 3))
    lam = np.empty(count)
    steps = np.empty(count, dtype=np.int64)
    for b in range(count):
        while True:
            d = rng.uniform(size=6)
            wl = (0.05 + 1.95 * d[0], -1.0 + 2.0 * d[1], 0.05 + 1.95 * d[2])
            wr = (0.05 + 1.95 * d[3], -1.0 + 2.0 * d[4], 0.05 + 1.95 * d[5])
            if not riemann.has_vacuum(GAMMA, wl, wr):
                break
        left[b], right[b] = wl, wr
        dx = 1.0 / lengths[b]
        lam[b], steps[b] = _round_lambda(LAMBDA_FACTOR[lattice] * lambda_1d_riemann(GAMMA, wl, wr), dx, t_final)
    return TubeBatch(lengths, left, right, lam, steps, t_final, omega, lattice=lattice)


# --------------------------------------------------------------------------- 2-D

def _cell_centres(n, x0, dx):
    return x0 + (np.arange(n) + 0.5) * dx


def _quadrant_fields(nx, ny, dx, x0, y0, xc, yc, q):
    x = _cell_centres(nx, x0, dx)[None, :]
    y = _cell_centres(ny, y0, dx)[:, None]
    right, top = x >= xc, y >= yc
    prim = np.empty((4, ny, nx))
    for k in range(4):
        prim[k] = np.where(top, np.where(right, q[1][k], q[2][k]), np.where(right, q[4][k], q[3][k]))
    return prim


def quadrant_riemann(seed: int = 0, n: int = 1024, omega: float = 1.0, steps: int = 1000) -> Workload2D:
    """Seeded four-quadrant 2-D Riemann problem on [0, 1]^2, split at (0.5, 0.5).

    Quadrant states: rho ~ U[0.1, 1.5], p ~ U[0.03, 1.5], u, v ~ U[-1.2, 1.2].
    A draw for which any of the four interface Riemann problems generates
    vacuum is replaced by the next draw.  Transmissive boundaries all round.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        d = rng.uniform(size=(4, 4))
        q = {i + 1: (0.1 + 1.4 * d[i, 0], -1.2 + 2.4 * d[i, 1], -1.2 + 2.4 * d[i, 2], 0.03 + 1.47 * d[i, 3])
             for i in range(4)}
        ok = True
        for a, b in ((2, 1), (3, 4)):
            ok &= not riemann.has_vacuum(GAMMA, (q[a][0], q[a][1], q[a][3]), (q[b][0], q[b][1], q[b][3]))
        for a, b in ((4, 1), (3, 2)):
            ok &= not riemann.has_vacuum(GAMMA, (q[a][0], q[a][2], q[a][3]), (q[b][0], q[b][2], q[b][3]))
        if ok:
            break
    dx = 1.0 / n
    prim = _quadrant_fields(n, n, dx, 0.0, 0.0, 0.5, 0.5, q)
    lam = lambda_2d_quadrants(GAMMA, q)
    return Workload2D(f"quadrant_riemann_s{seed}", n, n, dx, 0.0, 0.0, prim, [("transmissive", None)] * 4,
                      lam, omega, steps, meta={"quadrants": q, "seed": seed})


def paper_riemann_case4(n: int = 400, omega: float = 1.0, steps: int = 100) -> Workload2D:
    """The paper's 2-D Riemann problem (Liska-Wendroff case 4), Section III.

    The paper writes the quadrants around the origin while solving on
    [0, 1]^2; they are placed here around the centre (0.5, 0.5).
    """
    q = {1: (1.1, 0.0, 0.0, 1.1), 2: (0.5065, 0.8939, 0.0, 0.35),
         3: (1.1, 0.8939, 0.8939, 1.1), 4: (0.5065, 0.0, 0.8939, 0.35)}
    dx = 1.0 / n
    prim = _quadrant_fields(n, n, dx, 0.0, 0.0, 0.5, 0.5, q)
    lam = lambda_2d_quadrants(GAMMA, q)
    return Workload2D("paper_riemann_case4", n, n, dx, 0.0, 0.0, prim, [("transmissive", None)] * 4,
                      lam, omega, steps, meta={"quadrants": q})


def explosion(n: int = 400, omega: float = 1.0, steps: int = 100) -> Workload2D:
    """Cylindrical explosion on [-1, 1]^2: (1, 0, 0, 1) inside r < 0.4, (0.125, 0, 0, 0.1) outside."""
    dx = 2.0 / n
    x = _cell_centres(n, -1.0, dx)[None, :]
    y = _cell_centres(n, -1.0, dx)[:, None]
    inside = x * x + y * y < 0.16
    prim = np.empty((4, n, n))
    for k, (a, b) in enumerate(zip((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1))):
        prim[k] = np.where(inside, a, b)
    lam = 1.1 * max(bouchut_speed(GAMMA, *s) for s in
                    [(1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1)] +
                    [(r, u, 0.0, p) for (r, u, p) in
                     riemann.star_states(GAMMA, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))])
    return Workload2D("explosion", n, n, dx, -1.0, -1.0, prim, [("transmissive", None)] * 4, lam, omega, steps)


OBLIQUE_INFLOW = (1.0, 2.9, 0.0, 1.0 / 1.4)
OBLIQUE_BETA_DEG = 29.0


def oblique_shock_reflection(nx: int = 4096, ny: int = 1024, omega: float = 1.0,
                             steps: int = 20000, top_state=None) -> Workload2D:
    """Oblique shock reflection on [0, 4] x [0, 1] (Section III).

    Inflow (1, 2.9, 0, 1/1.4) on the left; the top held at the state behind a
    29-degree oblique shock; free-slip wall at the bottom; transmissive
    outflow on the right; interior initialised to the inflow state.
    """
    dx = 4.0 / nx
    if abs(dx - 1.0 / ny) > 1e-15:
        raise ValueError("D2Q4 needs dx == dy: use nx = 4 ny")
    inflow = OBLIQUE_INFLOW
    top = top_state or post_shock_state(GAMMA, inflow[0], inflow[1], inflow[3], OBLIQUE_BETA_DEG)
    prim = np.empty((4, ny, nx))
    for k in range(4):
        prim[k] = inflow[k]
    lam = 1.1 * max(bouchut_speed(GAMMA, *inflow), bouchut_speed(GAMMA, *top))
    bc = [("dirichlet", inflow), ("transmissive", None), ("wall", None), ("dirichlet", tuple(top))]
    return Workload2D("oblique_shock", nx, ny, dx, 0.0, 0.0, prim, bc, lam, omega, steps,
                      meta={"top": tuple(top)})


def uniform_2d(nx, ny, state=(1.0, 0.5, 0.3, 1.0), bc="periodic", lam=None, omega=1.0, steps=10) -> Workload2D:
    """Uniform flow; every boundary of the given kind (Dirichlet at the same state)."""
    prim = np.empty((4, ny, nx))
    for k in range(4):
        prim[k] = state[k]
    lam = lam or 1.2 * bouchut_speed(GAMMA, *state)
    b = (bc, tuple(state) if bc == "dirichlet" else None)
    return Workload2D("uniform", nx, ny, 1.0 / nx, 0.0, 0.0, prim, [b] * 4, lam, omega, steps)


def adjoint_pulses(seed: int = 0, n: int = 2048, pulses: int = 8, amp: float = 0.1, width: float = 0.05,
                   omega: float = 1.0, steps: int = 2000, lam: float = 3.0):
    """Uniform flow (1, 0.5, 0.3, 1) plus seeded Gaussian pulses in rho and p, periodic [0, 1]^2.

    Returns (workload, rho_target) where the target density is 1 plus pulses
    drawn from seed + 1.  Distances use the periodic minimum image.
    """
    def pulses_field(rng):
        c = rng.uniform(size=(pulses, 2))
        x = _cell_centres(n, 0.0, 1.0 / n)
        f = np.zeros((n, n))
        for cx, cy in c:
            dxp = np.abs(x - cx)
            dxp = np.minimum(dxp, 1.0 - dxp)
            dyp = np.abs(x - cy)
            dyp = np.minimum(dyp, 1.0 - dyp)
            f += amp * np.exp(-(dyp[:, None] ** 2 + dxp[None, :] ** 2) / (2.0 * width ** 2))
        return f

    base = (1.0, 0.5, 0.3, 1.0)
    bump = pulses_field(np.random.Generator(np.random.PCG64(seed)))
    prim = np.empty((4, n, n))
    prim[0] = base[0] + bump
    prim[1] = base[1]
    prim[2] = base[2]
    prim[3] = base[3] + bump
    target = 1.0 + pulses_field(np.random.Generator(np.random.PCG64(seed + 1)))
    wl = Workload2D(f"adjoint_pulses_s{seed}", n, n, 1.0 / n, 0.0, 0.0, prim, [("periodic", None)] * 4,
                    lam, omega, steps)
    return wl, target


# ---------------------------------------------------------------- internal walls

FFS_INFLOW = (1.4, 3.0, 0.0, 1.0)          # Mach 3: a = sqrt(1.4 * 1 / 1.4) = 1


def normal_shock_state(gamma, rho1, u1, p1, mach):
    """State behind a normal shock of Mach number `mach` relative to a gas (rho1, u1, p1)
    moving along +x; the shock moves along +x (Rankine-Hugoniot, ideal gas).
    Returns (rho2, u2, p2) in the frame of the input state."""
    a1 = sound(gamma, rho1, p1)
    m2 = mach * mach
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    w = u1 + mach * a1                      # shock speed
    u2 = w - (w - u1) * rho1 / rho2         # mass flux continuity in the shock frame
    return rho2, u2, p2


def forward_facing_step(nx: int = 240, ny: int = 80, omega: float = 1.0, t_final: float = 4.0,
                        steps: int | None = None, lam_factor: float = 1.5) -> Workload2D:
    """Mach 3 flow over a forward-facing step in the channel [0, 3] x [0, 1] (Section III).

    The step is the block x >= 0.6, y < 0.2 (solid cells).  Inflow (1.4, 3, 0, 1) on the
    left, transmissive outflow on the right, free-slip walls at the bottom and the top;
    the interior starts at the inflow state.  lambda = lam_factor times the D2Q4 bound of the
    stagnation state behind the bow shock (the largest bound the run meets, checked by the
    oracle), raised so that t_final is a whole number of steps.
    """
    dx = 3.0 / nx
    if abs(dx - 1.0 / ny) > 1e-15:
        raise ValueError("D2Q4 needs dx == dy: use nx = 3 ny")
    x = _cell_centres(nx, 0.0, dx)[None, :]
    y = _cell_centres(ny, 0.0, dx)[:, None]
    solid = ((x >= 0.6) & (y < 0.2)).astype(np.uint8)
    prim = np.empty((4, ny, nx))
    for k in range(4):
        prim[k] = FFS_INFLOW[k]
    rho, u, v, p = FFS_INFLOW
    mach = u / sound(GAMMA, rho, p)
    r2, u2_lab, p2 = normal_shock_state(GAMMA, rho, 0.0, p, mach)
    u2 = mach * sound(GAMMA, rho, p) - u2_lab                   # behind a standing normal shock
    lam0 = max(bouchut_speed(GAMMA, rho, u, v, p), bouchut_speed(GAMMA, r2, u2, 0.0, p2),
               bouchut_speed(GAMMA, r2, 0.0, u2, p2))
    lam = lam_factor * lam0
    if steps is None:
        lam, steps = _round_lambda(lam, dx, t_final)
    bc = [("dirichlet", FFS_INFLOW), ("transmissive", None), ("wall", None), ("wall", None)]
    return Workload2D("forward_facing_step", nx, ny, dx, 0.0, 0.0, prim, bc, lam, omega, int(steps),
                      meta={"step": (0.6, 0.2), "t_final": t_final}, solid=solid)


def shock_diffraction(n: int = 400, omega: float = 1.0, t_final: float = 0.1561, steps: int | None = None,
                      corner=(0.1, 0.6), mach: float = 5.09, lam_factor: float = 2.0) -> Workload2D:
    """A Mach 5.09 normal shock diffracting over a backward-facing step in [0, 1]^2 (Section III).

    The step is the block x < corner[0], y < corner[1] (solid cells).  The shock starts at
    x = corner[0] above the step, moving along +x into gas at rest (1.4, 0, 0, 1); behind it
    the Rankine-Hugoniot state.  Left side: that state (inflow); right and top transmissive;
    bottom a free-slip wall.  lambda = lam_factor times the D2Q4 bound of the post-shock
    state (the corner expansion accelerates the flow; checked by the oracle).
    """
    dx = 1.0 / n
    xs, ys = corner
    x = _cell_centres(n, 0.0, dx)[None, :]
    y = _cell_centres(n, 0.0, dx)[:, None]
    solid = ((x < xs) & (y < ys)).astype(np.uint8)
    pre = (1.4, 0.0, 0.0, 1.0)
    r2, u2, p2 = normal_shock_state(GAMMA, pre[0], pre[1], pre[3], mach)
    post = (r2, u2, 0.0, p2)
    prim = np.empty((4, n, n))
    behind = np.broadcast_to(x < xs, (n, n))
    for k in range(4):
        prim[k] = np.where(behind, post[k], pre[k])
    lam = lam_factor * bouchut_speed(GAMMA, *post)
    if steps is None:
        lam, steps = _round_lambda(lam, dx, t_final)
    bc = [("dirichlet", post), ("transmissive", None), ("wall", None), ("transmissive", None)]
    return Workload2D("shock_diffraction", n, n, dx, 0.0, 0.0, prim, bc, lam, omega, int(steps),
                      meta={"corner": corner, "mach": mach, "post": post, "t_final": t_final}, solid=solid)


# ---------------------------------------------------------------- scalar 2-D Burgers

BURGERS_CASES = {
    # (u at x = 0, u at x = 1, bottom profile u(x, 0) = b0 + b1 x)        (Section III)
    1: (1.0, -1.0, (1.0, -2.0)),
    2: (1.5, -0.5, (1.5, -2.0)),
}


def burgers_2d(case: int = 1, n: int = 64, omega: float = 1.0, t_final: float = 3.0, steps: int | None = None,
               safety: float = 1.1) -> Workload2D:
    """The 2-D inviscid Burgers problems of Section III on [0, 1]^2, u_t + (u^2/2)_x + u_y = 0.

    Dirichlet u = left / right values on x = 0, 1 and the linear profile on y = 0; the top
    is an outflow (transmissive; the y-speed g2' = 1 carries everything out).  The interior
    starts at the bottom profile extended in y.  lambda = safety * max(|u| + 1) over the
    boundary data (the scalar D2Q4 bound |g1'| + |g2'|), rounded so that t_final is a whole
    number of steps.  The steady state is reached after a few crossing times (t = 3).
    """
    left, right, (b0, b1) = BURGERS_CASES[case]
    dx = 1.0 / n
    x = _cell_centres(n, 0.0, dx)[None, :]
    prim = np.broadcast_to(b0 + b1 * x, (n, n))[None].copy()
    umax = max(abs(left), abs(right), abs(b0), abs(b0 + b1))
    lam = safety * (umax + 1.0)
    if steps is None:
        lam, steps = _round_lambda(lam, dx, t_final)
    bc = [("dirichlet", (left, 0.0, 0.0, 0.0)), ("dirichlet", (right, 0.0, 0.0, 0.0)),
          ("dirichlet", (b0, b1, 0.0, 0.0)), ("transmissive", None)]
    return Workload2D(f"burgers_case{case}", n, n, dx, 0.0, 0.0, prim, bc, lam, omega, int(steps),
                      meta={"case": case, "t_final": t_final}, law="burgers")


def burgers_steady_exact(case: int, x, y):
    """Exact steady solution of the Section III Burgers problems (characteristics dx/dy = u).

    Below y = 1/2 the bottom characteristics fan in towards the focus: u = (b0 + b1 x) along
    x = x0 + u y gives u = (b0 + b1 x) / (1 + b1 y) between the lines carrying the left and
    right boundary values; above it a shock moves with slope (u_l + u_r) / 2 from the focus.
    """
    left, right, (b0, b1) = BURGERS_CASES[case]
    x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
    below = y < 0.5
    fan = (b0 + b1 * x) / (1.0 + b1 * y)
    xl = left * y                          # the characteristic from (0, 0) carrying u = left
    xr = 1.0 + right * y                   # the one from (1, 0) carrying u = right
    u_below = np.where(x <= xl, left, np.where(x >= xr, right, fan))
    xf = left * 0.5                        # the focus (the fan's lines all meet at y = 1/2)
    xs = xf + 0.5 * (left + right) * (y - 0.5)
    u_above = np.where(x < xs, left, right)
    return np.where(below, u_below, u_above)


# --------------------------------------------------------------------------- seeded configurations

CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")
CONFIG_NAMES = ("sod_d1q2_1000", "quadrant_riemann_1024", "oblique_shock_4096x1024", "batched_tubes_4096",
                "adjoint_pulses_2048")


def load_config(name: str) -> dict:
    """The seeded configuration `name` (a JSON file under workloads/configs/)."""
    with open(os.path.join(CONFIG_DIR, name + ".json")) as fh:
        return json.load(fh)


def from_config(name: str, **overrides):
    """(configuration, workload) of a seeded configuration; keyword overrides replace its kwargs
    (e.g. a shorter step count for a bounded sample)."""
    cfg = load_config(name)
    kwargs = dict(cfg["kwargs"], **overrides)
    return cfg, globals()[cfg["generator"]](**kwargs)

