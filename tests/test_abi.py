"""CPU checks of the C ABI: the library loads, exports every declared symbol,
its structures match the header byte for byte, and invalid calls fail with
the documented status before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbrs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1504_07034_gb300.build import build
    build()
    from paper_1504_07034_gb300 import abi
    return abi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbrs_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    from paper_1504_07034_gb300 import abi
    for name in names:
        assert hasattr(lib, name), f"liblbrs.so does not export {name}"
        assert name in abi.SIGNATURES, f"binding lacks {name}"


def test_struct_layout_matches_header(tmp_path):
    from paper_1504_07034_gb300 import abi
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "lbrs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lbrs_config), offsetof(lbrs_config, nx),
         offsetof(lbrs_config, gamma), offsetof(lbrs_config, dx), offsetof(lbrs_config, bc),
         offsetof(lbrs_config, cuda_stream), sizeof(lbrs_bc), sizeof(lbrs_diag));
  printf("%zu %zu\n", offsetof(lbrs_diag, max_lambda_local), offsetof(lbrs_diag, n_subchar));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    C, D = abi.lbrs_config, abi.lbrs_diag
    want = [ctypes.sizeof(C), C.nx.offset, C.gamma.offset, C.dx.offset, C.bc.offset, C.cuda_stream.offset,
            ctypes.sizeof(abi.lbrs_bc), ctypes.sizeof(D), D.max_lambda_local.offset, D.n_subchar.offset]
    assert got == want


def _cfg(**kw):
    from paper_1504_07034_gb300.solver import make_config
    args = dict(gamma=1.4, lam=3.0, omega=1.0, dx=1 / 64, bc=[("transmissive", None)] * 4, precision="f32",
                stream_handle=0)
    lattice = kw.pop("lattice", "d2q4")
    nx, ny = kw.pop("nx", 64), kw.pop("ny", 64)
    args.update(kw)
    return make_config(lattice, nx, ny, **args)


def test_workspace_size_formula(lib):
    from paper_1504_07034_gb300 import abi
    size = ctypes.c_size_t()
    cfg = _cfg(nx=1024, ny=1024)
    assert lib.lbrs_workspace_size(ctypes.byref(cfg), ctypes.byref(size)) == abi.LBRS_OK
    f_bytes = 16 * 1024 * 1024 * 4
    assert 2 * f_bytes <= size.value < 2 * f_bytes + 64 * 1024
    cfg64 = _cfg(nx=1000, ny=1, lattice="d1q2", precision="f64", bc=[("transmissive", None)] * 2)
    assert lib.lbrs_workspace_size(ctypes.byref(cfg64), ctypes.byref(size)) == abi.LBRS_OK
    assert size.value >= 2 * 6 * 1000 * 8


@pytest.mark.parametrize("bad,needle", [
    (dict(omega=2.0), "omega"),
    (dict(omega=0.0), "omega"),
    (dict(lam=-1.0), "lambda"),
    (dict(gamma=1.0), "gamma"),
    (dict(dx=0.0), "dx"),
    (dict(nx=0), "nx"),
    (dict(lattice="d1q2", ny=4, bc=[("transmissive", None)] * 2), "ny == 1"),
    (dict(bc=[("wall", None), ("transmissive", None), ("transmissive", None), ("transmissive", None)]), "wall"),
    (dict(bc=[("periodic", None), ("transmissive", None), ("transmissive", None), ("transmissive", None)]), "periodic"),
    (dict(bc=[("dirichlet", (-1.0, 0, 0, 1)), ("transmissive", None), ("transmissive", None), ("transmissive", None)]), "Dirichlet"),
    (dict(ny=1, bc=[("transmissive", None), ("transmissive", None), ("wall", None), ("transmissive", None)]), "ny >= 2"),
    (dict(lattice="d2q4s", bc=[("transmissive", None)] * 2 + [("wall", None)] * 2), "wall"),
    (dict(lattice="d2q4s", bc=[("dirichlet", (float("nan"), 0.0))] + [("transmissive", None)] * 3), "profile"),
    (dict(lattice="d2q4s", precision="f16neq"), "D2Q4 storage forms"),
])
def test_invalid_config_rejected(lib, bad, needle):
    from paper_1504_07034_gb300 import abi
    cfg = _cfg(**bad)
    size = ctypes.c_size_t(123)
    st = lib.lbrs_workspace_size(ctypes.byref(cfg), ctypes.byref(size))
    assert st == abi.LBRS_EINVAL
    assert size.value == 123
    assert needle in lib.lbrs_last_error(None).decode()


def test_struct_size_guard(lib):
    from paper_1504_07034_gb300 import abi
    cfg = _cfg()
    cfg.struct_size = 8
    assert lib.lbrs_workspace_size(ctypes.byref(cfg), ctypes.byref(ctypes.c_size_t())) == abi.LBRS_EINVAL


def test_create_argument_errors_without_device_work(lib):
    from paper_1504_07034_gb300 import abi
    cfg = _cfg()
    ctx = ctypes.c_void_p()
    assert lib.lbrs_create(ctypes.byref(cfg), None, 1 << 30, ctypes.byref(ctx)) == abi.LBRS_EINVAL
    assert lib.lbrs_create(ctypes.byref(cfg), ctypes.c_void_p(0x1008), 1 << 30, ctypes.byref(ctx)) == abi.LBRS_EINVAL
    assert "aligned" in lib.lbrs_last_error(None).decode()
    assert lib.lbrs_create(ctypes.byref(cfg), ctypes.c_void_p(0x10000), 16, ctypes.byref(ctx)) == abi.LBRS_ENOMEM
    assert ctx.value is None


def test_null_context_calls(lib):
    from paper_1504_07034_gb300 import abi
    assert lib.lbrs_step(None, 1) == abi.LBRS_EINVAL
    assert lib.lbrs_sync(None) == abi.LBRS_EINVAL
    assert lib.lbrs_moments(None, None, 1, 0) == abi.LBRS_EINVAL
    assert lib.lbrs_set_state(None, None, 1, 0, 0) == abi.LBRS_EINVAL
    lib.lbrs_destroy(None)
    assert lib.lbrs_status_string(abi.LBRS_ESUBCHAR) == b"LBRS_ESUBCHAR"
    assert lib.lbrs_abi_version() == abi.ABI_VERSION


def test_scalar_lattice_workspace(lib):
    """The scalar D2Q4 lattice stores 4 populations of one field per cell; Dirichlet profiles may
    take any finite value and slope (a negative u is a valid state of the scalar law)."""
    from paper_1504_07034_gb300 import abi
    bc = [("dirichlet", (-1.0, 2.0)), ("dirichlet", (1.5, -0.5)), ("transmissive", None), ("transmissive", None)]
    cfg = _cfg(lattice="d2q4s", nx=100, ny=30, bc=bc, precision="f64")
    size = ctypes.c_size_t()
    assert lib.lbrs_workspace_size(ctypes.byref(cfg), ctypes.byref(size)) == abi.LBRS_OK
    assert 2 * 4 * 100 * 30 * 8 <= size.value < 2 * 4 * 100 * 30 * 8 + 64 * 1024
