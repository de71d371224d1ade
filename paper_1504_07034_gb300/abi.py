"""ctypes binding of the C ABI in include/lbrs.h (argument marshalling only).

Every function keeps its C name (``lbrs_create``, ``lbrs_step`` ...) and
signature; structures mirror the header field for field.  All computation
happens in liblbrs.so.  Loading fails loudly if the library has not been
built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "liblbrs.so"

# enums (include/lbrs.h)
LBRS_OK, LBRS_EINVAL, LBRS_ENOMEM, LBRS_ECUDA, LBRS_ENONPHYS, LBRS_ESUBCHAR, LBRS_ETIMEOUT, LBRS_ESTATE = range(8)
LBRS_D1Q2, LBRS_D2Q4, LBRS_D1Q3, LBRS_D2Q4S = 0, 1, 2, 3
LBRS_F64, LBRS_F32, LBRS_F16NEQ, LBRS_F32U = 0, 1, 2, 3
LBRS_BC_PERIODIC, LBRS_BC_TRANSMISSIVE, LBRS_BC_DIRICHLET, LBRS_BC_WALL, LBRS_BC_CUT, LBRS_BC_WALL_HALFWAY = range(6)
LBRS_CONSERVED, LBRS_PRIMITIVE = 0, 1
ABI_VERSION = 1

BC_KINDS = {"periodic": LBRS_BC_PERIODIC, "transmissive": LBRS_BC_TRANSMISSIVE,
            "dirichlet": LBRS_BC_DIRICHLET, "wall": LBRS_BC_WALL, "cut": LBRS_BC_CUT,
            "wall_halfway": LBRS_BC_WALL_HALFWAY}


class lbrs_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("halo_rows", ctypes.c_int32), ("prim", ctypes.c_double * 4)]


class lbrs_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("lattice", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("diag_every", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("gamma", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("bc", lbrs_bc * 4),
        ("cuda_stream", ctypes.c_void_p),
    ]


class lbrs_diag(ctypes.Structure):
    _fields_ = [
        ("totals", ctypes.c_double * 4),
        ("min_rho", ctypes.c_double),
        ("min_p", ctypes.c_double),
        ("max_lambda_local", ctypes.c_double),
        ("reserved", ctypes.c_double),
        ("n_nonphysical", ctypes.c_int64),
        ("n_subchar", ctypes.c_int64),
    ]


class lbrs_batch_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("lattice", ctypes.c_int32),
        ("batch", ctypes.c_int64),
        ("lengths", ctypes.POINTER(ctypes.c_int64)),
        ("lam", ctypes.POINTER(ctypes.c_double)),
        ("gamma", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
    ]


class lbrs_batch_tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("cells_per_thread", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_CTX = ctypes.c_void_p
SIGNATURES = {
    "lbrs_abi_version": (ctypes.c_int, []),
    "lbrs_debug_build": (ctypes.c_int, []),
    "lbrs_selftest_wait_timeout": (ctypes.c_int, [_CTX]),
    "lbrs_selftest_rcp_f32": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "lbrs_debug_check": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
    "lbrs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lbrs_workspace_size": (ctypes.c_int, [ctypes.POINTER(lbrs_config), ctypes.POINTER(ctypes.c_size_t)]),
    "lbrs_create": (ctypes.c_int, [ctypes.POINTER(lbrs_config), _P, ctypes.c_size_t, ctypes.POINTER(_CTX)]),
    "lbrs_destroy": (None, [_CTX]),
    "lbrs_set_state": (ctypes.c_int, [_CTX, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbrs_step": (ctypes.c_int, [_CTX, ctypes.c_int64]),
    "lbrs_sync": (ctypes.c_int, [_CTX]),
    "lbrs_first_bad_step": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbrs_moments": (ctypes.c_int, [_CTX, _P, ctypes.c_int, ctypes.c_int]),
    "lbrs_diagnostics": (ctypes.c_int, [_CTX, ctypes.POINTER(lbrs_diag)]),
    "lbrs_boundary_flux": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "lbrs_diagnostics_noalloc": (ctypes.c_int, [ctypes.POINTER(lbrs_config), _P, ctypes.POINTER(lbrs_diag)]),
    "lbrs_get_distributions": (ctypes.c_int, [_CTX, _P, ctypes.c_int]),
    "lbrs_set_distributions": (ctypes.c_int, [_CTX, _P, ctypes.c_int, ctypes.c_int64]),
    "lbrs_set_obstacles": (ctypes.c_int, [_CTX, _P]),
    "lbrs_checkpoint_size": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_size_t)]),
    "lbrs_checkpoint_save": (ctypes.c_int, [_CTX, _P, ctypes.c_int]),
    "lbrs_checkpoint_load": (ctypes.c_int, [_CTX, _P, ctypes.c_int]),
    "lbrs_step_adaptive": (ctypes.c_int, [_CTX, ctypes.c_int64, ctypes.c_double, ctypes.c_double]),
    "lbrs_adaptive_state": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    "lbrs_halo_size": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_size_t)]),
    "lbrs_halo_export": (ctypes.c_int, [_CTX, ctypes.c_int, _P, ctypes.c_int]),
    "lbrs_halo_import": (ctypes.c_int, [_CTX, ctypes.c_int, _P, ctypes.c_int]),
    "lbrs_store_rows": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "lbrs_rows_export": (ctypes.c_int, [_CTX, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int]),
    "lbrs_rows_import": (ctypes.c_int, [_CTX, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int]),
    "lbrs_step_count": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbrs_launch_count": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbrs_last_error": (ctypes.c_char_p, [_CTX]),
    "lbrs_step_record": (ctypes.c_int, [_CTX, ctypes.c_int64, _P]),
    "lbrs_adjoint_seed": (ctypes.c_int, [_CTX, _P, ctypes.c_int, _P]),
    "lbrs_vjp_loss": (ctypes.c_int, [_CTX, _P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "lbrs_adjoint_step": (ctypes.c_int, [_CTX, _P, _P, _P]),
    "lbrs_vjp_equilibrium": (ctypes.c_int, [_CTX, _P, _P, _P]),
    "lbrs_adjoint_workspace_size": (ctypes.c_int, [_CTX, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "lbrs_forward_checkpointed": (ctypes.c_int, [_CTX, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_size_t]),
    "lbrs_backward_checkpointed": (ctypes.c_int, [_CTX, _P, _P, _P]),
    "lbrs_batch_workspace_size": (ctypes.c_int, [ctypes.POINTER(lbrs_batch_config), ctypes.POINTER(ctypes.c_size_t)]),
    "lbrs_batch_create": (ctypes.c_int, [ctypes.POINTER(lbrs_batch_config), _P, ctypes.c_size_t, ctypes.POINTER(_CTX)]),
    "lbrs_batch_destroy": (None, [_CTX]),
    "lbrs_batch_set_state": (ctypes.c_int, [_CTX, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbrs_batch_run": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbrs_batch_moments": (ctypes.c_int, [_CTX, _P, ctypes.c_int, ctypes.c_int]),
    "lbrs_batch_get_distributions": (ctypes.c_int, [_CTX, _P, ctypes.c_int]),
    "lbrs_batch_get_tuning": (ctypes.c_int, [_CTX, ctypes.POINTER(lbrs_batch_tuning)]),
    "lbrs_batch_set_tuning": (ctypes.c_int, [_CTX, ctypes.POINTER(lbrs_batch_tuning)]),
    "lbrs_batch_autotune": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(lbrs_batch_tuning),
                                           ctypes.POINTER(ctypes.c_double)]),
    "lbrs_batch_launch_count": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbrs_batch_last_error": (ctypes.c_char_p, [_CTX]),
}

_lib = None


class LbrsError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{status_name(status)}: {message}")


def library_path() -> Path:
    return Path(os.environ.get("LBRS_LIBRARY", LIB_PATH))


def load():
    """Load liblbrs.so (built by paper_1504_07034_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not path.exists():
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -m paper_1504_07034_gb300.build); there is no CPU fallback")
        lib = ctypes.CDLL(str(path))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if lib.lbrs_abi_version() != ABI_VERSION:
            raise RuntimeError("liblbrs.so ABI version mismatch")
        _lib = lib
    return _lib


def status_name(status: int) -> str:
    names = ["LBRS_OK", "LBRS_EINVAL", "LBRS_ENOMEM", "LBRS_ECUDA", "LBRS_ENONPHYS", "LBRS_ESUBCHAR",
             "LBRS_ETIMEOUT", "LBRS_ESTATE"]
    return names[status] if 0 <= status < len(names) else f"status {status}"


def check(status: int, ctx=None):
    if status != LBRS_OK:
        msg = load().lbrs_last_error(ctx)
        raise LbrsError(status, (msg or b"").decode())
    return status


def __getattr__(name):
    """Module-level access to the C functions by their C names: abi.lbrs_step(ctx, n)."""
    if name.startswith("lbrs_") and name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
