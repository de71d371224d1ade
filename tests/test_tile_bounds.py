"""Bounds of the direct-offset (interior) path of the kernels with a tile-height parameter, on the CPU.

The scalar two-step kernel (step2ds_fused2_kernel) and the adjoint's 4-field sweep (adj_fused2_u_kernel)
load the window of an interior tile on direct offsets, without wrapping or clamping.  For every tile height
the launcher accepts, every tile the launch grid holds and a spread of grid sizes, each load of such a
tile must stay inside the grid.  The interior predicate, the window's cell formula, the load offsets, the
window size and the accepted heights are read from the kernel source, so the check follows the code.
"""
import itertools
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1504_07034_gb300", "csrc", "lbrs_kernels_f32.cu")

KERNELS = {
    # kernel: its launcher
    "step2ds_fused2_kernel": "launch_step2s_f32",
    "adj_fused2_u_kernel": "launch_adj_fused2_u_f32",
}


@pytest.fixture(scope="module")
def src():
    with open(SRC) as f:
        return f.read()


def _body(src, head):
    i = src.index(head)
    return src[i:src.index("\n}\n", i)]


def _c_to_py(expr):
    assert re.fullmatch(r"[A-Za-z0-9_ .+\-*/%<>=&()]+", expr), expr
    return expr.replace("&&", " and ").replace("a.nx", "nx").replace("a.ny", "ny").replace("/", "//")


def _kernel(src, name):
    body = _body(src, f" {name}(")
    const = {"kFTX": int(re.search(r"\bkFTX = (\d+)", src).group(1)),
             "kFWX": None}
    const["kFWX"] = eval(re.search(r"\bkFWX = ([^,;]+)[,;]", src).group(1), {}, const)
    inside = _c_to_py(re.search(r"const bool inside = (.+?);", body).group(1))
    m = re.search(r"\(int64_t\)\((j0 - 1 \+ w / kFWX)\) \* a\.nx \+ \((i0 - 1 \+ w % kFWX)\)", body)
    assert m, f"window cell formula of {name} not found"
    row, col = _c_to_py(m.group(1)), _c_to_py(m.group(2))
    m = re.search(r"const int64_t (?:src|s)\[4\] = \{([^}]*)\}", body)
    assert m, f"load offsets of {name} not found"
    offsets = []
    big = 1 << 20
    for e in m.group(1).split(","):
        v = eval(_c_to_py(e.strip()), {"__builtins__": {}}, {"c": 0, "nx": big})
        dy = round(v / big)
        offsets.append((v - dy * big, dy))
    assert all(abs(dx) == 1 and abs(dy) == 1 for dx, dy in offsets), offsets
    twn = _c_to_py(re.search(r"constexpr int kTWN = ([^;]+);", body).group(1))
    launcher = _body(src, f"cudaError_t {KERNELS[name]}(")
    allowed = [int(x) for x in re.search(r"allowed\[\] = \{([^}]*)\}", launcher).group(1).split(",")]
    assert allowed[-1] == 0
    return dict(const=const, inside=inside, row=row, col=col, offsets=offsets, twn=twn, heights=allowed[:-1])


@pytest.mark.parametrize("name", sorted(KERNELS))
def test_interior_loads_stay_in_the_grid(src, name):
    k = _kernel(src, name)
    assert k["heights"], name
    for ty in k["heights"]:
        env0 = dict(k["const"], TY=ty)
        twn = eval(k["twn"], {"__builtins__": {}}, env0)
        interior_tiles = 0
        for nx, ny in itertools.product((34, 35, 36, 66, 67, 68, 99, 100, 130),
                                        (ty + 2, ty + 3, ty + 4, 2 * ty + 3, 2 * ty + 4, 3 * ty + 5, 80, 81)):
            for i0, j0 in itertools.product(range(0, nx, 32), range(0, ny, ty)):   # the launch grid's tiles
                env = dict(env0, nx=nx, ny=ny, i0=i0, j0=j0)
                if not eval(k["inside"], {"__builtins__": {}}, env):
                    continue
                interior_tiles += 1
                for w in range(twn):
                    env["w"] = w
                    y = eval(k["row"], {"__builtins__": {}}, env)
                    x = eval(k["col"], {"__builtins__": {}}, env)
                    for dx, dy in k["offsets"]:
                        assert 0 <= x + dx < nx and 0 <= y + dy < ny, (name, ty, nx, ny, i0, j0, w, dx, dy)
                # the tile's own cells, which phase 2 stores, lie in the grid too
                assert i0 + env0["kFTX"] <= nx and j0 + ty <= ny
        assert interior_tiles > 0, (name, ty)


@pytest.mark.parametrize("name", sorted(KERNELS))
def test_window_covers_tile_and_halo(src, name):
    """The window is the tile plus one cell on every side: kFWX = tile width + 2, kTWN = kFWX (TY + 2)."""
    k = _kernel(src, name)
    for ty in k["heights"]:
        env = dict(k["const"], TY=ty)
        assert k["const"]["kFWX"] == k["const"]["kFTX"] + 2
        assert eval(k["twn"], {"__builtins__": {}}, env) == (k["const"]["kFTX"] + 2) * (ty + 2)
