"""Python face of the LBRS solver: torch tensors in, C ABI calls out.

``Solver`` owns a torch uint8 workspace on the GPU (PyTorch is only the
allocator and the stream provider here) and a context of liblbrs.so.  Every
step of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import abi

_DTYPE_CODE = {torch.float64: abi.LBRS_F64, torch.float32: abi.LBRS_F32,
               np.dtype(np.float64): abi.LBRS_F64, np.dtype(np.float32): abi.LBRS_F32}
_PRECISION = {"f64": abi.LBRS_F64, "f32": abi.LBRS_F32, "f16neq": abi.LBRS_F16NEQ, "f32u": abi.LBRS_F32U}


def make_config(lattice: str, nx: int, ny: int, *, gamma: float, lam: float, omega: float, dx: float,
                bc, precision: str, stream_handle: int, diag_every: int = 0) -> abi.lbrs_config:
    cfg = abi.lbrs_config()
    cfg.struct_size = ctypes.sizeof(abi.lbrs_config)
    cfg.lattice = {"d2q4": abi.LBRS_D2Q4, "d2q4s": abi.LBRS_D2Q4S, "d1q2": abi.LBRS_D1Q2,
                   "d1q3": abi.LBRS_D1Q3}[lattice]
    cfg.precision = _PRECISION[precision]
    cfg.diag_every = int(diag_every)
    cfg.nx, cfg.ny = int(nx), int(ny)
    cfg.gamma, cfg.lam, cfg.omega, cfg.dx = float(gamma), float(lam), float(omega), float(dx)
    for s, (kind, state) in enumerate(bc):
        cfg.bc[s].kind = abi.BC_KINDS[kind]
        if kind == "cut":                        # state: the ghost rows stored beyond the cut (None: 2)
            cfg.bc[s].halo_rows = int(state or 0)
            continue
        if state is not None:
            for k, v in enumerate(state):
                cfg.bc[s].prim[k] = float(v)
    cfg.cuda_stream = stream_handle or None
    return cfg


class Solver:
    """One LBRS problem on one GPU.

    lattice   "d1q2", "d1q3", "d2q4" or "d2q4s" (the scalar 2-D Burgers law; one field u; a
              Dirichlet side's state is the linear profile (value, slope) along it)
    bc        per side (x-lo, x-hi[, y-lo, y-hi]): (kind, primitive_state_or_None); a y side
              ("cut", rows_or_None) makes the solver one y-slab of a larger grid (halo_export/import)
    precision "f64" (plain FP64 path), "f32" (FP32 distributions), "f16neq" (D2Q4: FP32
              moments plus FP16 non-equilibrium parts) or "f32u" (D2Q4 at omega = 1: FP32 moments only)
    stream    a torch.cuda.Stream (default: the current stream)
    """

    def __init__(self, lattice: str, nx: int, ny: int = 1, *, lam: float, dx: float, bc, gamma: float = 1.4,
                 omega: float = 1.0, precision: str = "f32", stream: torch.cuda.Stream | None = None,
                 device: torch.device | str | None = None, diag_every: int = 0):
        self.lib = abi.load()
        self.solid = None
        self.lattice = lattice
        self.Q, self.K = {"d2q4": (4, 4), "d2q4s": (4, 1), "d1q2": (2, 3), "d1q3": (3, 3)}[lattice]
        self.nx, self.ny = int(nx), int(ny)
        self.precision = precision
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        sides = 4 if lattice in ("d2q4", "d2q4s") else 2
        bc = list(bc)
        if len(bc) < sides:
            raise ValueError(f"need {sides} boundary conditions")
        bc = bc + [("periodic", None)] * (4 - len(bc))
        self.cfg = make_config(lattice, nx, ny, gamma=gamma, lam=lam, omega=omega, dx=dx, bc=bc,
                               precision=precision, stream_handle=self.stream.cuda_stream, diag_every=diag_every)
        size = ctypes.c_size_t()
        abi.check(self.lib.lbrs_workspace_size(ctypes.byref(self.cfg), ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            abi.check(self.lib.lbrs_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                           size.value, ctypes.byref(ctx)))
        self.ctx = ctx
        ny_s, row0 = ctypes.c_int64(), ctypes.c_int64()
        abi.check(self.lib.lbrs_store_rows(ctx, ctypes.byref(ny_s), ctypes.byref(row0)))
        self.ny_store, self.row0 = ny_s.value, row0.value   # stored rows (a cut context adds ghost rows)

    @classmethod
    def from_workload(cls, wl, precision: str = "f32", stream=None, omega=None, diag_every: int = 0,
                      lattice: str = "d1q2"):
        if hasattr(wl, "ny"):
            lat = "d2q4s" if getattr(wl, "law", "euler") == "burgers" else "d2q4"
            s = cls(lat, wl.nx, wl.ny, lam=wl.lam, dx=wl.dx, bc=wl.bc, gamma=wl.gamma,
                    omega=wl.omega if omega is None else omega, precision=precision, stream=stream,
                    diag_every=diag_every)
            if getattr(wl, "solid", None) is not None:
                s.set_obstacles(torch.from_numpy(wl.solid))
            return s
        return cls(lattice, wl.nx, 1, lam=wl.lam, dx=wl.dx, bc=wl.bc, gamma=wl.gamma,
                   omega=wl.omega if omega is None else omega, precision=precision, stream=stream,
                   diag_every=diag_every)

    # ------------------------------------------------------------------ helpers
    @property
    def grid(self):
        return (self.ny, self.nx) if self.lattice in ("d2q4", "d2q4s") else (self.nx,)

    @property
    def storage_dtype(self):
        return torch.float64 if self.precision == "f64" else torch.float32

    def _check(self, status):
        return abi.check(status, self.ctx)

    def raw_state(self) -> torch.Tensor:
        """The storage buffer as bytes (any precision): lbrs_get_distributions into a uint8 tensor."""
        n = self.nx * self.ny
        nbytes = {"f16neq": n * 40 + 16, "f32u": n * 16}.get(
            self.precision, self.Q * self.K * n * (8 if self.precision == "f64" else 4))
        out = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._check(self.lib.lbrs_get_distributions(self.ctx, ctypes.c_void_p(out.data_ptr()), 1))
        return out

    def set_raw_state(self, raw: torch.Tensor, step: int = 0):
        self._check(self.lib.lbrs_set_distributions(self.ctx, ctypes.c_void_p(raw.data_ptr()), 1 if raw.is_cuda else 0,
                                                    int(step)))

    # ------------------------------------------------------------------ C ABI calls
    def set_state(self, W, primitive: bool = True):
        """f = f^eq(U0); W of shape (K, *grid): torch tensor (GPU or CPU) or numpy array."""
        kind = abi.LBRS_PRIMITIVE if primitive else abi.LBRS_CONSERVED
        if isinstance(W, np.ndarray):
            W = np.ascontiguousarray(W)
            if W.dtype not in (np.float64, np.float32):
                W = W.astype(np.float64)
            if W.shape != (self.K,) + self.grid:
                raise ValueError(f"expected shape {(self.K,) + self.grid}, got {W.shape}")
            self._check(self.lib.lbrs_set_state(self.ctx, ctypes.c_void_p(W.ctypes.data), 0,
                                                _DTYPE_CODE[W.dtype], kind))
            return
        if tuple(W.shape) != (self.K,) + self.grid:
            raise ValueError(f"expected shape {(self.K,) + self.grid}, got {tuple(W.shape)}")
        if W.dtype not in (torch.float64, torch.float32):
            raise TypeError("W must be float64 or float32")
        W = W.contiguous()
        on_dev = 1 if W.is_cuda else 0
        self._check(self.lib.lbrs_set_state(self.ctx, ctypes.c_void_p(W.data_ptr()), on_dev, _DTYPE_CODE[W.dtype],
                                            kind))
        self._keep = W  # device input stays referenced until the next call

    def step(self, n: int = 1):
        self._check(self.lib.lbrs_step(self.ctx, int(n)))

    def sync(self):
        self._check(self.lib.lbrs_sync(self.ctx))

    def first_bad_step(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.lbrs_first_bad_step(self.ctx, ctypes.byref(v)))
        return v.value

    def moments(self, dtype=torch.float64, out: torch.Tensor | None = None) -> torch.Tensor:
        """Conserved fields U (K, *grid); on the GPU unless `out` is a CPU tensor."""
        if out is None:
            out = torch.empty((self.K,) + self.grid, dtype=dtype, device=self.device)
        if tuple(out.shape) != (self.K,) + self.grid or not out.is_contiguous():
            raise ValueError("out must be a contiguous (K, *grid) tensor")
        self._check(self.lib.lbrs_moments(self.ctx, ctypes.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0,
                                          _DTYPE_CODE[out.dtype]))
        return out

    def diagnostics(self) -> dict:
        d = abi.lbrs_diag()
        st = self.lib.lbrs_diagnostics(self.ctx, ctypes.byref(d))
        if st not in (abi.LBRS_OK, abi.LBRS_ENONPHYS, abi.LBRS_ESUBCHAR):
            self._check(st)
        return {"status": abi.status_name(st), "totals": [d.totals[k] for k in range(self.K)],
                "min_rho": d.min_rho, "min_p": d.min_p, "max_lambda_local": d.max_lambda_local,
                "n_nonphysical": d.n_nonphysical, "n_subchar": d.n_subchar}

    def boundary_flux(self) -> dict:
        """FP64 per-field sums (times dx^2) of what the next step brings in across the domain's
        sides and takes out (lbrs_boundary_flux): totals after one step = totals + inflow - outflow."""
        fin = (ctypes.c_double * 4)()
        fout = (ctypes.c_double * 4)()
        self._check(self.lib.lbrs_boundary_flux(self.ctx, fin, fout))
        return {"inflow": [fin[k] for k in range(self.K)], "outflow": [fout[k] for k in range(self.K)]}

    def get_distributions(self, out: torch.Tensor | None = None) -> torch.Tensor:
        """The raw state.  For the reduced storage forms (f16neq: U and the FP16
        non-equilibrium parts; f32u: U) it fills only the leading bytes of the
        (Q, K, *grid) tensor; a tensor allocated here is zero beyond them."""
        if out is None:
            alloc = torch.empty if self.precision in ("f64", "f32") else torch.zeros
            out = alloc((self.Q, self.K) + self.grid, dtype=self.storage_dtype, device=self.device)
        if out.dtype != self.storage_dtype or not out.is_contiguous() or out.numel() != self.Q * self.K * self.nx * self.ny:
            raise ValueError("out must be a contiguous (Q, K, *grid) tensor of the storage dtype")
        self._check(self.lib.lbrs_get_distributions(self.ctx, ctypes.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0))
        return out

    def set_distributions(self, f: torch.Tensor, step: int = 0):
        if f.dtype != self.storage_dtype or not f.is_contiguous() or f.numel() != self.Q * self.K * self.nx * self.ny:
            raise ValueError("f must be a contiguous (Q, K, *grid) tensor of the storage dtype")
        self._check(self.lib.lbrs_set_distributions(self.ctx, ctypes.c_void_p(f.data_ptr()), 1 if f.is_cuda else 0,
                                                    int(step)))

    # ------------------------------------------------------------------ y-slabs (cut sides)
    def halo_size(self, side: int) -> tuple[int, int]:
        """(ghost rows, bytes of one exchanged block) of y side 2 (y-lo) or 3 (y-hi)."""
        rows, nbytes = ctypes.c_int64(), ctypes.c_size_t()
        self._check(self.lib.lbrs_halo_size(self.ctx, int(side), ctypes.byref(rows), ctypes.byref(nbytes)))
        return rows.value, nbytes.value

    def halo_buffer(self, side: int, device=None) -> torch.Tensor:
        """An empty (P, rows, nx) tensor of the storage dtype for one exchanged block."""
        rows, _ = self.halo_size(side)
        planes = 4 if self.precision == "f32u" else self.Q * self.K
        return torch.empty((planes, rows, self.nx), dtype=self.storage_dtype,
                           device=self.device if device is None else device)

    def halo_export(self, side: int, out: torch.Tensor) -> torch.Tensor:
        """The own rows next to cut `side`, every plane, into `out` (from halo_buffer)."""
        self._check(self.lib.lbrs_halo_export(self.ctx, int(side), ctypes.c_void_p(out.data_ptr()),
                                              1 if out.is_cuda else 0))
        return out

    def halo_import(self, side: int, block: torch.Tensor):
        """The neighbour's exported block into the ghost rows beyond cut `side`."""
        self._keep_halo = getattr(self, "_keep_halo", {})
        self._keep_halo[side] = block                       # referenced until the next import of this side
        self._check(self.lib.lbrs_halo_import(self.ctx, int(side), ctypes.c_void_p(block.data_ptr()),
                                              1 if block.is_cuda else 0))

    def checkpoint(self, device: bool = True) -> torch.Tensor:
        """The state as a self-describing blob (uint8 tensor on the GPU, or in pinned host memory)."""
        size = ctypes.c_size_t()
        self._check(self.lib.lbrs_checkpoint_size(self.ctx, ctypes.byref(size)))
        blob = torch.empty(size.value, dtype=torch.uint8, device=self.device if device else "cpu")
        self._check(self.lib.lbrs_checkpoint_save(self.ctx, ctypes.c_void_p(blob.data_ptr()), 1 if device else 0))
        return blob

    def restore(self, blob: torch.Tensor):
        """Resume from a blob of checkpoint(); the configuration must match."""
        blob = blob.contiguous()
        self._check(self.lib.lbrs_checkpoint_load(self.ctx, ctypes.c_void_p(blob.data_ptr()), 1 if blob.is_cuda else 0))

    def step_adaptive(self, n: int, safety: float = 1.0, t_final: float = 0.0):
        """n steps with the lattice speed chosen anew every step (see lbrs_step_adaptive)."""
        self._check(self.lib.lbrs_step_adaptive(self.ctx, int(n), float(safety), float(t_final)))

    def adaptive_state(self) -> dict:
        t, lam, steps, done = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int()
        self._check(self.lib.lbrs_adaptive_state(self.ctx, ctypes.byref(t), ctypes.byref(lam), ctypes.byref(steps),
                                                 ctypes.byref(done)))
        return {"t": t.value, "lambda": lam.value, "steps": steps.value, "done": bool(done.value)}

    def run_to_time(self, t_final: float, safety: float = 1.0, chunk: int = 64, max_steps: int = 10 ** 8) -> dict:
        """Adaptive steps until t_final is reached exactly, enqueued `chunk` at a time (one
        synchronisation per chunk); returns the adaptive state at the end."""
        st = self.adaptive_state()
        while not st["done"] and st["steps"] < max_steps:
            self.step_adaptive(chunk, safety, t_final)
            st = self.adaptive_state()
        return st

    def set_obstacles(self, solid):
        """Internal walls from a (ny, nx) mask (nonzero = solid cell); None removes them.
        The mask is kept on the device for the solver's lifetime (the library reads it
        at every step)."""
        if solid is None:
            self._check(self.lib.lbrs_set_obstacles(self.ctx, None))
            self.solid = None
            return
        m = torch.as_tensor(solid).to(device=self.device, dtype=torch.uint8).contiguous()
        if tuple(m.shape) != (self.ny, self.nx):
            raise ValueError(f"obstacle mask must have shape {(self.ny, self.nx)}")
        self._check(self.lib.lbrs_set_obstacles(self.ctx, ctypes.c_void_p(m.data_ptr())))
        self.solid = m

    # ------------------------------------------------------------------ adjoint (periodic D2Q4)
    @property
    def store_grid(self):
        """Grid of the adjoint buffers: the stored rows (own rows plus the ghost rows of cuts)."""
        return (self.ny_store, self.nx) if self.lattice in ("d2q4", "d2q4s") else (self.nx,)

    def _fields_tensor(self, n=None):
        shape = ((n,) if n is not None else ()) + (self.K,) + self.store_grid
        return torch.empty(shape, dtype=self.storage_dtype, device=self.device)

    def _dists_tensor(self):
        return torch.empty((self.Q, self.K) + self.store_grid, dtype=self.storage_dtype, device=self.device)

    def own_rows(self, t: torch.Tensor) -> torch.Tensor:
        """The own rows of a stored-layout tensor (..., ny_store, nx)."""
        return t[..., self.row0:self.row0 + self.ny, :]

    def rows_export(self, side: int, buf: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """The own rows next to cut `side` of a stored-layout tensor, all its planes, into `out`
        (planes x ghost rows x nx)."""
        planes = buf.numel() // (self.ny_store * self.nx)
        self._check(self.lib.lbrs_rows_export(self.ctx, int(side), self._ptr(buf), planes,
                                              ctypes.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0))
        return out

    def rows_import(self, side: int, buf: torch.Tensor, block: torch.Tensor):
        """The neighbour's block into the ghost rows beyond cut `side` of a stored-layout tensor."""
        planes = buf.numel() // (self.ny_store * self.nx)
        self._keep_rows = block
        self._check(self.lib.lbrs_rows_import(self.ctx, int(side), self._ptr(buf), planes,
                                              ctypes.c_void_p(block.data_ptr()), 1 if block.is_cuda else 0))

    @staticmethod
    def _ptr(t: torch.Tensor):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("expected a contiguous CUDA tensor")
        return ctypes.c_void_p(t.data_ptr())

    def step_record(self, n: int, U_hist: torch.Tensor | None = None) -> torch.Tensor:
        """n steps, returning the moments each step's collision used: (n, K, *grid)."""
        U_hist = self._fields_tensor(n) if U_hist is None else U_hist
        self._check(self.lib.lbrs_step_record(self.ctx, int(n), self._ptr(U_hist)))
        return U_hist

    def adjoint_seed(self, dLdU: torch.Tensor) -> torch.Tensor:
        g = self._dists_tensor()
        dLdU = dLdU.contiguous()
        self._check(self.lib.lbrs_adjoint_seed(self.ctx, self._ptr(dLdU), _DTYPE_CODE[dLdU.dtype], self._ptr(g)))
        return g

    def vjp_loss(self, rho_target: torch.Tensor):
        """(L, dL/df*) of L = 1/2 sum (rho - rho_target)^2 dx^d for the current state."""
        g = self._dists_tensor()
        rho_target = rho_target.contiguous()
        loss = ctypes.c_double()
        self._check(self.lib.lbrs_vjp_loss(self.ctx, self._ptr(rho_target), _DTYPE_CODE[rho_target.dtype],
                                           self._ptr(g), ctypes.byref(loss)))
        return loss.value, g

    def adjoint_step(self, U_next: torch.Tensor, gbar: torch.Tensor, out: torch.Tensor | None = None):
        out = self._dists_tensor() if out is None else out
        self._check(self.lib.lbrs_adjoint_step(self.ctx, self._ptr(U_next), self._ptr(gbar), self._ptr(out)))
        return out

    def vjp_equilibrium(self, U0: torch.Tensor, gbar0: torch.Tensor) -> torch.Tensor:
        grad = self._fields_tensor()
        self._check(self.lib.lbrs_vjp_equilibrium(self.ctx, self._ptr(U0), self._ptr(gbar0), self._ptr(grad)))
        return grad

    def forward_checkpointed(self, n_steps: int, segment: int | None = None):
        """n_steps with checkpoints every `segment` steps (default ceil(sqrt(n_steps)))."""
        import math
        segment = int(segment or math.ceil(math.sqrt(n_steps)))
        size = ctypes.c_size_t()
        self._check(self.lib.lbrs_adjoint_workspace_size(self.ctx, int(n_steps), segment, ctypes.byref(size)))
        self.adj_ws = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self._check(self.lib.lbrs_forward_checkpointed(self.ctx, int(n_steps), segment,
                                                       self._ptr(self.adj_ws), size.value))
        return self.adj_ws

    def backward_checkpointed(self, gbar_T: torch.Tensor) -> torch.Tensor:
        grad = self._fields_tensor()
        self._check(self.lib.lbrs_backward_checkpointed(self.ctx, self._ptr(self.adj_ws), self._ptr(gbar_T),
                                                        self._ptr(grad)))
        return grad

    @property
    def step_count(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.lbrs_step_count(self.ctx, ctypes.byref(v)))
        return v.value

    @property
    def launch_count(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.lbrs_launch_count(self.ctx, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbrs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent D1Q2 tubes (uneven lengths, per-tube lambda) on one GPU.

    lengths, lam  per-tube cell counts and lattice speeds
    boundary      "transmissive" or "periodic" (both ends of every tube)
    The state is concatenated: fields (3, sum N), tube b at offsets[b].
    """

    def __init__(self, lengths, lam, *, gamma: float = 1.4, omega: float = 1.0, boundary: str = "transmissive",
                 precision: str = "f32", stream: torch.cuda.Stream | None = None, lattice: str = "d1q2"):
        self.lib = abi.load()
        self.lattice = lattice
        self.Q = {"d1q2": 2, "d1q3": 3}[lattice]
        self.lengths = np.ascontiguousarray(lengths, dtype=np.int64)
        self.lam = np.ascontiguousarray(lam, dtype=np.float64)
        self.batch = len(self.lengths)
        self.N = int(self.lengths.sum())
        self.offsets = np.concatenate([[0], np.cumsum(self.lengths)[:-1]]).astype(np.int64)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfg = abi.lbrs_batch_config()
        cfg.struct_size = ctypes.sizeof(abi.lbrs_batch_config)
        cfg.precision = _PRECISION[precision]
        cfg.boundary = abi.BC_KINDS[boundary]
        cfg.lattice = abi.LBRS_D1Q3 if lattice == "d1q3" else abi.LBRS_D1Q2
        cfg.batch = self.batch
        cfg.lengths = self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        cfg.lam = self.lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.gamma, cfg.omega = float(gamma), float(omega)
        cfg.cuda_stream = self.stream.cuda_stream or None
        self.cfg = cfg
        size = ctypes.c_size_t()
        abi.check(self.lib.lbrs_batch_workspace_size(ctypes.byref(cfg), ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        abi.check(self.lib.lbrs_batch_create(ctypes.byref(cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                             size.value, ctypes.byref(ctx)))
        self.ctx = ctx

    @classmethod
    def from_tubes(cls, tubes, precision: str = "f32", stream=None, lattice: str | None = None):
        return cls(tubes.lengths, tubes.lam, gamma=tubes.gamma, omega=tubes.omega, precision=precision,
                   stream=stream, lattice=lattice or getattr(tubes, "lattice", "d1q2"))

    @property
    def storage_dtype(self):
        return torch.float64 if self.precision == "f64" else torch.float32

    def _check(self, status):
        if status != abi.LBRS_OK:
            msg = self.lib.lbrs_batch_last_error(self.ctx) if self.ctx else b""
            raise abi.LbrsError(status, (msg or b"").decode())

    def set_state(self, W, primitive: bool = True):
        kind = abi.LBRS_PRIMITIVE if primitive else abi.LBRS_CONSERVED
        if isinstance(W, np.ndarray):
            W = torch.from_numpy(np.ascontiguousarray(W))
        if tuple(W.shape) != (3, self.N):
            raise ValueError(f"expected shape (3, {self.N}), got {tuple(W.shape)}")
        W = W.contiguous()
        self._check(self.lib.lbrs_batch_set_state(self.ctx, ctypes.c_void_p(W.data_ptr()), 1 if W.is_cuda else 0,
                                                  _DTYPE_CODE[W.dtype], kind))
        self._keep = W

    def run(self, steps):
        steps = np.ascontiguousarray(steps, dtype=np.int64)
        if steps.shape != (self.batch,):
            raise ValueError("steps must have one entry per tube")
        self._check(self.lib.lbrs_batch_run(self.ctx, steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))

    def moments(self, dtype=torch.float64, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((3, self.N), dtype=dtype, device=self.device)
        self._check(self.lib.lbrs_batch_moments(self.ctx, ctypes.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0,
                                                _DTYPE_CODE[out.dtype]))
        return out

    def get_distributions(self) -> torch.Tensor:
        out = torch.empty((self.Q, 3, self.N), dtype=self.storage_dtype, device=self.device)
        self._check(self.lib.lbrs_batch_get_distributions(self.ctx, ctypes.c_void_p(out.data_ptr()), 1))
        return out

    @property
    def tuning(self):
        t = abi.lbrs_batch_tuning()
        self._check(self.lib.lbrs_batch_get_tuning(self.ctx, ctypes.byref(t)))
        return (t.block, t.cells_per_thread, t.halo)

    @tuning.setter
    def tuning(self, value):
        t = abi.lbrs_batch_tuning(*value, 0)
        self._check(self.lib.lbrs_batch_set_tuning(self.ctx, ctypes.byref(t)))

    def autotune(self, steps):
        steps = np.ascontiguousarray(steps, dtype=np.int64)
        t = abi.lbrs_batch_tuning()
        ns = ctypes.c_double()
        self._check(self.lib.lbrs_batch_autotune(self.ctx, steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                 ctypes.byref(t), ctypes.byref(ns)))
        return (t.block, t.cells_per_thread, t.halo), ns.value

    @property
    def launch_count(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.lbrs_batch_launch_count(self.ctx, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbrs_batch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
