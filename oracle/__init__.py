"""Plain FP64 CPU oracle of the LBRS time step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and to time against.  The
product path (``paper_1504_07034_gb300``) never imports it, and the two share
no code.  The arithmetic lives in ``lbrs_oracle.c`` (plain C, float64, no FMA
contraction, OpenMP over rows); this module only compiles it and marshals
numpy arrays through ctypes.

Array layout: distributions ``fs[q, k, j, i]`` (2-D) or ``fs[q, k, i]`` (1-D),
conserved fields ``U[k, j, i]`` / ``U[k, i]``.  Lattice velocity order
follows the paper: D1Q2 (-lambda, +lambda); D1Q3 (-lambda, 0, +lambda);
D2Q4 f1..f4 with signs (-,-), (+,-), (+,+), (-,+).

Every function is pinned by ``tests/test_oracle_pins.py`` against what the
paper and the mathematics fix (moment identities, the exact Lax-Friedrichs
form at omega = 1, uniform-flow and contact invariants, conservation,
mirror symmetries, the exact Riemann solution, the Chapman-Enskog diffusion
rate, the wall relations, brute force on tiny grids).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lbrs_oracle.c"
LIB = HERE / "_build" / "liblbrs_oracle.so"

BC_KINDS = {"periodic": 0, "transmissive": 1, "dirichlet": 2, "wall": 3, "wall_halfway": 4}
D1Q2, D1Q3, D2Q4, D2Q4S = 2, 3, 4, 5      # D2Q4S: the scalar 2-D inviscid Burgers law


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no FMA contraction; OpenMP).

    The environment variable LBRS_ORACLE_LIB points the module at another
    compiled copy instead (the mutation tests use it to load deliberately
    broken oracles and check that the pins catch them).
    """
    alt = os.environ.get("LBRS_ORACLE_LIB")
    if alt:
        return Path(alt)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    LIB.parent.mkdir(parents=True, exist_ok=True)
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           str(SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("nthreads", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("gamma", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("bc_kind", ctypes.c_int32 * 4),
        ("bc_prim", (ctypes.c_double * 4) * 4),
        ("solid", ctypes.POINTER(ctypes.c_uint8)),
        ("dx", ctypes.c_double),
    ]


class _Check(ctypes.Structure):
    _fields_ = [
        ("first_bad_step", ctypes.c_int64),
        ("n_nonphysical", ctypes.c_int64),
        ("n_subchar", ctypes.c_int64),
        ("max_lambda_local", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_prim_to_cons.argtypes = [P, dp, dp]
        L.orc_cons_to_prim.argtypes = [P, dp, dp]
        L.orc_feq.argtypes = [P, ctypes.c_int64, dp, dp]
        L.orc_init.argtypes = [P, dp, dp]
        L.orc_moments.argtypes = [P, dp, dp]
        L.orc_validate.argtypes = [P]
        L.orc_validate.restype = ctypes.c_int
        L.orc_stream.argtypes = [P, dp, dp]
        L.orc_stream.restype = ctypes.c_int
        L.orc_collide.argtypes = [P, dp, dp, dp, ctypes.POINTER(_Check), ctypes.c_int64]
        L.orc_run.argtypes = [P, dp, dp, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(_Check)]
        L.orc_run.restype = ctypes.c_int
        L.orc_totals.argtypes = [P, dp, ctypes.c_double, dp]
        L.orc_boundary_flux.argtypes = [P, dp, dp, ctypes.c_double, dp, dp]
        L.orc_boundary_flux.restype = ctypes.c_int
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_adjoint_step.argtypes = [P, dp, dp, dp]
        L.orc_adjoint_step.restype = ctypes.c_int
        L.orc_vjp_equilibrium.argtypes = [P, dp, dp, dp]
        L.orc_vjp_equilibrium.restype = ctypes.c_int
        L.orc_run_adaptive.argtypes = [P, dp, dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       dp, dp, dp]
        L.orc_run_adaptive.restype = ctypes.c_int64
        L.orc_obstacle_check.argtypes = [P]
        L.orc_obstacle_check.restype = ctypes.c_int64
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(lib().orc_max_threads())


class Oracle:
    """One LBRS problem: lattice, grid, gamma, lambda, omega, boundary conditions."""

    def __init__(self, lattice: int, nx: int, ny: int = 1, *, gamma: float = 1.4, lam: float,
                 omega: float = 1.0, bc=None, nthreads: int = 0, solid=None, dx: float = 1.0):
        self.lattice = lattice
        self.Q, self.K = {D2Q4: (4, 4), D2Q4S: (4, 1), D1Q3: (3, 3), D1Q2: (2, 3)}[lattice]
        self.nx, self.ny = int(nx), int(ny)
        sides = 4 if lattice in (D2Q4, D2Q4S) else 2
        bc = list(bc) if bc is not None else [("periodic", None)] * sides
        if len(bc) != sides:
            raise ValueError(f"need {sides} boundary conditions")
        p = _Params()
        p.lattice, p.nthreads = lattice, nthreads
        p.nx, p.ny = self.nx, self.ny
        p.gamma, p.lam, p.omega = gamma, lam, omega
        p.dx = dx
        for s, (kind, state) in enumerate(bc):
            p.bc_kind[s] = BC_KINDS[kind]
            if state is not None:
                for k, val in enumerate(state):
                    p.bc_prim[s][k] = float(val)
        self.solid = None
        if solid is not None:
            self.solid = np.ascontiguousarray(solid, dtype=np.uint8)
            if self.solid.shape != (self.ny, self.nx):
                raise ValueError(f"solid mask must have shape {(self.ny, self.nx)}")
            p.solid = self.solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        self.p = p
        err = lib().orc_validate(ctypes.byref(p))
        if err:
            raise ValueError(f"invalid oracle parameters (code {err})")
        if lib().orc_obstacle_check(ctypes.byref(p)):
            raise ValueError("obstacle geometry leaves a fluid cell without a known mirror population")

    @classmethod
    def from_workload(cls, wl, nthreads: int = 0, omega=None, lattice=None):
        if hasattr(wl, "ny"):
            law = D2Q4S if getattr(wl, "law", "euler") == "burgers" else D2Q4
            return cls(lattice or law, wl.nx, wl.ny, gamma=wl.gamma, lam=wl.lam,
                       omega=wl.omega if omega is None else omega, bc=wl.bc, nthreads=nthreads,
                       solid=getattr(wl, "solid", None), dx=wl.dx)
        return cls(lattice or D1Q2, wl.nx, 1, gamma=wl.gamma, lam=wl.lam,
                   omega=wl.omega if omega is None else omega, bc=wl.bc, nthreads=nthreads)

    # shapes -------------------------------------------------------------
    @property
    def grid(self):
        return (self.ny, self.nx) if self.lattice in (D2Q4, D2Q4S) else (self.nx,)

    def _fields(self, a) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.K,) + self.grid:
            raise ValueError(f"expected shape {(self.K,) + self.grid}, got {a.shape}")
        return a

    def _dists(self, a) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.Q, self.K) + self.grid:
            raise ValueError(f"expected shape {(self.Q, self.K) + self.grid}, got {a.shape}")
        return a

    # operations ----------------------------------------------------------
    def prim_to_cons(self, W) -> np.ndarray:
        W = self._fields(W)
        U = np.empty_like(W)
        lib().orc_prim_to_cons(ctypes.byref(self.p), _ptr(W), _ptr(U))
        return U

    def cons_to_prim(self, U) -> np.ndarray:
        U = self._fields(U)
        W = np.empty_like(U)
        lib().orc_cons_to_prim(ctypes.byref(self.p), _ptr(U), _ptr(W))
        return W

    def feq(self, U) -> np.ndarray:
        """Equilibria of arbitrary states U[K, ...] -> feq[Q, K, ...]."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        shape = U.shape[1:]
        n = int(np.prod(shape)) if shape else 1
        out = np.empty((self.Q, self.K) + shape)
        lib().orc_feq(ctypes.byref(self.p), n, _ptr(U), _ptr(out))
        return out

    def init(self, U0) -> np.ndarray:
        U0 = self._fields(U0)
        fs = np.empty((self.Q, self.K) + self.grid)
        lib().orc_init(ctypes.byref(self.p), _ptr(U0), _ptr(fs))
        return fs

    def stream(self, fs) -> np.ndarray:
        """Streaming plus boundary conditions (the streamed f before collision)."""
        fs = self._dists(fs)
        f = np.empty_like(fs)
        err = lib().orc_stream(ctypes.byref(self.p), _ptr(fs), _ptr(f))
        if err:
            raise ValueError(f"oracle stream error {err}")
        return f

    def collide(self, f, step: int = 0):
        """Returns (fs, U, check) for a streamed f."""
        f = self._dists(f)
        fs = np.empty_like(f)
        U = np.empty((self.K,) + self.grid)
        chk = _Check(-1, 0, 0, 0.0)
        lib().orc_collide(ctypes.byref(self.p), _ptr(f), _ptr(fs), _ptr(U), ctypes.byref(chk), step)
        return fs, U, _check_dict(chk)

    def run(self, fs, nsteps: int, step0: int = 0):
        """Advance a copy of fs by nsteps steps. Returns (fs, check)."""
        fs = self._dists(fs).copy()
        work = np.empty_like(fs)
        chk = _Check(-1, 0, 0, 0.0)
        err = lib().orc_run(ctypes.byref(self.p), _ptr(fs), _ptr(work), int(nsteps), int(step0),
                            ctypes.byref(chk))
        if err:
            raise ValueError(f"oracle run error {err}")
        return fs, _check_dict(chk)

    def run_adaptive(self, fs, nsteps: int, dx: float, safety: float, t_final: float = 0.0):
        """Advance a copy of fs (whose equilibria were built with this problem's lambda) with
        the lambda chosen anew every step: each step streams with the current state's lambda
        (advancing dx / lambda) and collides with safety times the largest local bound of the
        state before it and of the Dirichlet states; stop at t_final exactly if positive.
        Returns (fs, the stream lambda of every step, time reached, lambda of the final state)."""
        fs = self._dists(fs).copy()
        work = np.empty_like(fs)
        lam = np.empty(max(int(nsteps), 1))
        t, lam_next = ctypes.c_double(), ctypes.c_double()
        n = lib().orc_run_adaptive(ctypes.byref(self.p), _ptr(fs), _ptr(work), int(nsteps), float(dx),
                                   float(safety), float(t_final), _ptr(lam), ctypes.byref(t), ctypes.byref(lam_next))
        if n < 0:
            raise ValueError(f"oracle adaptive run error {n}")
        return fs, lam[:n].copy(), t.value, lam_next.value

    def moments(self, fs) -> np.ndarray:
        fs = self._dists(fs)
        U = np.empty((self.K,) + self.grid)
        lib().orc_moments(ctypes.byref(self.p), _ptr(fs), _ptr(U))
        return U

    def totals(self, fs, cell_volume: float) -> np.ndarray:
        fs = self._dists(fs)
        out = np.empty(self.K)
        lib().orc_totals(ctypes.byref(self.p), _ptr(fs), float(cell_volume), _ptr(out))
        return out

    def boundary_flux(self, fs, cell_volume: float):
        """(inflow, outflow) per field of the next step across the domain's sides (orc_boundary_flux)."""
        fs = self._dists(fs)
        work = np.empty_like(fs)
        fin, fout = np.empty(self.K), np.empty(self.K)
        err = lib().orc_boundary_flux(ctypes.byref(self.p), _ptr(fs), _ptr(work), float(cell_volume), _ptr(fin),
                                      _ptr(fout))
        if err:
            raise ValueError(f"oracle boundary flux error {err}")
        return fin, fout

    # adjoint (periodic D2Q4 only) ----------------------------------------
    def adjoint_step(self, U_next, gbar):
        """dL/dfs^n from gbar = dL/dfs^{n+1} and the moments U_next of step n+1."""
        U_next, gbar = self._fields(U_next), self._dists(gbar)
        out = np.empty_like(gbar)
        if lib().orc_adjoint_step(ctypes.byref(self.p), _ptr(U_next), _ptr(gbar), _ptr(out)):
            raise ValueError("the oracle adjoint covers periodic D2Q4 problems only")
        return out

    def vjp_equilibrium(self, U0, gbar0):
        """dL/dU0 = J_E(U0)^T gbar0 per cell."""
        U0, gbar0 = self._fields(U0), self._dists(gbar0)
        out = np.empty_like(U0)
        if lib().orc_vjp_equilibrium(ctypes.byref(self.p), _ptr(U0), _ptr(gbar0), _ptr(out)):
            raise ValueError("the oracle adjoint covers periodic D2Q4 problems only")
        return out

    def gradient(self, U0, nsteps: int, dLdU_T):
        """dL/dU0 for a loss L(U(T)) with dL/dU(T) given: forward storing every
        step's moments, then the backward sweep (plain full storage)."""
        fs = self.init(U0)
        Us = []
        for n in range(nsteps):
            f = self.stream(fs)
            fs, U, _ = self.collide(f, n + 1)
            Us.append(U)
        g = np.broadcast_to(np.asarray(dLdU_T)[None], (self.Q,) + np.shape(dLdU_T)).copy()
        for n in range(nsteps - 1, -1, -1):
            g = self.adjoint_step(Us[n], g)
        return self.vjp_equilibrium(U0, g), fs

    def timed_run(self, fs, nsteps: int):
        """Advance fs by nsteps and return (fs, seconds) measured around the step loop only."""
        fs = self._dists(fs).copy()
        work = np.empty_like(fs)
        chk = _Check(-1, 0, 0, 0.0)
        t0 = time.perf_counter()
        lib().orc_run(ctypes.byref(self.p), _ptr(fs), _ptr(work), int(nsteps), 0, ctypes.byref(chk))
        return fs, time.perf_counter() - t0


def _check_dict(c: _Check) -> dict:
    return {"first_bad_step": int(c.first_bad_step), "n_nonphysical": int(c.n_nonphysical),
            "n_subchar": int(c.n_subchar), "max_lambda_local": float(c.max_lambda_local)}
