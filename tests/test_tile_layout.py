"""The in-place windows of the two- and three-steps-per-launch kernels, checked on the CPU.

The FP32 two-step kernel (forward) and the FP32 two-step adjoint sweep fetch, per population q,
one tensor-copy box of 36 x 18 cells whose origin is shifted by that population's velocity, and
write the first step's result for each window slot over the box positions it read.  That is
hazard-free only if (a) the position a slot reads for population q holds exactly the cell the
method pulls from (forward: x - c_q; adjoint: x + c_q), (b) no two slots read the same position of
a population's box, (c) every position lies inside its box, (d) the second step reads population q
of its source slot at that slot's position, and (e) every box starts on a 16-byte boundary
(x times 4 bytes).  The box origins, the position rule and the second step's source slots are read
from the kernel source, so the test follows the code.  The three-step kernel (the last section) is
checked the same way over its three phases.
"""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1504_07034_gb300", "csrc", "lbrs_kernels_f32.cu")

# D2Q4 velocities in lattice units, populations in the paper's order (Section II.D)
SX = (-1, 1, 1, -1)
SY = (-1, -1, 1, 1)


@pytest.fixture(scope="module")
def src():
    with open(SRC) as f:
        return f.read()


def _const(src, name):
    m = re.search(rf"\b{name}\s*=\s*(\d+)", src)
    assert m, f"constant {name} not found"
    return int(m.group(1))


def _int_exprs(text, env):
    """Values of a brace list of small integer expressions such as {i0, i0 - 4, ti + 2}."""
    out = []
    for e in text.split(","):
        e = e.strip()
        assert re.fullmatch(r"[a-z0-9_ +\-]+", e), e
        out.append(eval(e, {"__builtins__": {}}, dict(env)))
    return out


def _array(src, fn, name, env):
    body = src[src.index(fn):]
    m = re.search(rf"const int {name}\[4\] = \{{([^}}]*)\}};", body)
    assert m, f"{name} of {fn} not found"
    return _int_exprs(m.group(1), env)


def _offset_rule(src, fn):
    """Populations whose position is shifted right by 2 in the box, from `(q == a || q == b) ? 2 : 0`."""
    body = src[src.index(fn):]
    m = re.search(r"\(\(q == (\d) \|\| q == (\d)\) \? 2 : 0\)", body)
    assert m, f"offset rule of {fn} not found"
    return {int(m.group(1)), int(m.group(2))}


KERNELS = {
    # name: (box-origin function, position function, second step's source slots, direction of the pull)
    "forward": ("void issue_tile_copy", "int tall_pos", "void tall_phase2", -1),
    "adjoint": ("void issue_adj_copy", "int adj_pos", "adj_fused2_tall_kernel", +1),
}


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_in_place_window(src, kernel):
    copy_fn, pos_fn, phase2_fn, sign = KERNELS[kernel]
    px, tx, ty = _const(src, "kPX"), _const(src, "kFTX"), _const(src, "kTY")
    wx, wy, py = tx + 2, ty + 2, ty + 2          # window 34 x 18, box 36 x 18
    shifted = _offset_rule(src, pos_fn)
    for i0 in (0, tx, 5 * tx):                   # tile origins: multiples of the tile width
        for j0 in (0, ty, 3 * ty):
            x0 = _array(src, copy_fn, "x0", {"i0": i0, "j0": j0})
            y0 = _array(src, copy_fn, "y0", {"i0": i0, "j0": j0})
            for q in range(4):
                assert (x0[q] * 4) % 16 == 0, (kernel, q, x0[q])              # (e)
                seen = set()
                for wj in range(wy):
                    for wi in range(wx):
                        # (a) the slot's global cell and the cell its population q comes from
                        x, y = i0 - 1 + wi, j0 - 1 + wj
                        sx, sy = x + sign * SX[q], y + sign * SY[q]
                        bx, by = sx - x0[q], sy - y0[q]
                        pos = (wj, wi + (2 if q in shifted else 0))
                        assert (by, bx) == pos, (kernel, q, wi, wj)
                        assert 0 <= bx < px and 0 <= by < py, (kernel, q, bx, by)  # (c)
                        assert pos not in seen                                     # (b)
                        seen.add(pos)


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_second_step_reads_where_the_first_wrote(src, kernel):
    """(d): interior tile cell (ti, tj) is window slot (ti + 1, tj + 1); population q of its second
    step comes from the cell x - c_q (forward) or x + c_q (adjoint), i.e. from window slot
    (ti + 1 -/+ sx_q, tj + 1 -/+ sy_q), which the kernel names in swi / swj."""
    _, _, phase2_fn, sign = KERNELS[kernel]
    tx, ty = _const(src, "kFTX"), _const(src, "kTY")
    for tj in range(ty):
        for ti in range(tx):
            swi = _array(src, phase2_fn, "swi", {"ti": ti, "tj": tj})
            swj = _array(src, phase2_fn, "swj", {"ti": ti, "tj": tj})
            for q in range(4):
                assert (swi[q], swj[q]) == (ti + 1 + sign * SX[q], tj + 1 + sign * SY[q]), (kernel, q)


# ---------------------------------------------------------------- the three-step kernel
#
# step2d_f32_fused3_kernel fetches, per population q, one box of kP3X x kW3Y cells (x from i0 - 4, y from
# the kernel's y0[q]) and works in place over three phases: phase 1 computes the kW3X x kW3Y window (tile
# plus two cells of halo) and writes each slot's population q over the position it pulled it from;
# phase 2 computes the kB3X x kB3Y inner slots, reading population q of source slot (u - sx, v - sy)
# where phase 1 left it and writing over that same position; phase 3 computes the tile, reading
# population q of inner slot (x - sx, y - sy) where phase 2 left it.  Hazard-free only if every position
# has one reader per phase and every read finds what the previous phase wrote there.

def _const_expr(src, name, env):
    m = re.search(rf"\b{name}\s*=\s*([A-Za-z0-9_ +*]+?)\s*[,;]", src)
    assert m, f"constant {name} not found"
    expr = m.group(1)
    assert re.fullmatch(r"[A-Za-z0-9_ +*]+", expr), expr
    return eval(expr, {"__builtins__": {}}, dict(env))


@pytest.fixture(scope="module")
def f3(src):
    return _f3_env(src)


def _f3_env(src):
    """The three-step kernel's constants, position offsets and box x origin, read from its source."""
    env = {}
    for name in ("kFTX", "kT3Y", "kT3T", "kP3X", "kW3X", "kW3Y", "kB3X", "kB3Y", "kP3N"):
        env[name] = _const_expr(src, name, env)
    body = src[src.index("int f3_pos("):]
    m = re.search(r"wj \* kP3X \+ wi \+ \(\(q == (\d) \|\| q == (\d)\) \? (\d) : (\d)\)", body)
    assert m, "position rule of f3_pos not found"
    a, b, hi, lo = (int(g) for g in m.groups())
    env["off"] = [hi if q in (a, b) else lo for q in range(4)]
    copy = src[src.index("void issue_tile_copy3("):]
    copy = copy[:copy.index("\n}")]
    mx = re.search(r'"r"\((i0 - \d+)\), "r"\(y0\[q\]\)', copy)
    assert mx, "x origin of issue_tile_copy3 not found"
    env["x0_expr"] = mx.group(1)
    env["y0_fn"] = "void issue_tile_copy3("
    pre = src[src.index("void prefetch_tile_l2_3("):]
    pre = pre[:pre.index("\n}")]
    mp = re.search(r'"r"\((i0 - \d+)\), "r"\(y0\[q\]\)', pre)
    assert mp, "x origin of prefetch_tile_l2_3 not found"
    env["prefetch_x0_expr"] = mp.group(1)
    return env


def test_three_step_boxes_hold_each_slots_pull(src, f3):
    """Phase 1: the position of slot (wi, wj), population q, holds the cell x - c_q; every position
    lies inside its box, no two slots share one, and every box starts on a 16-byte boundary."""
    e = f3
    assert e["kP3N"] == e["kP3X"] * e["kW3Y"]
    for i0 in (0, e["kFTX"], 7 * e["kFTX"]):
        for j0 in (0, e["kT3Y"], 5 * e["kT3Y"]):
            x0 = _int_exprs(e["x0_expr"], {"i0": i0, "j0": j0})[0]
            y0 = _array(src, e["y0_fn"], "y0", {"i0": i0, "j0": j0})
            assert (x0 * 4) % 16 == 0, x0
            # the L2 prefetch of a later tile asks for the same boxes
            assert _int_exprs(e["prefetch_x0_expr"], {"i0": i0})[0] == x0
            assert _array(src, "void prefetch_tile_l2_3(", "y0", {"i0": i0, "j0": j0}) == y0
            for q in range(4):
                seen = set()
                for wj in range(e["kW3Y"]):
                    for wi in range(e["kW3X"]):
                        col, row = wi + e["off"][q], wj
                        assert 0 <= col < e["kP3X"] and 0 <= row < e["kW3Y"], (q, wi, wj)
                        cell = (i0 - 2 + wi, j0 - 2 + wj)
                        assert (x0 + col, y0[q] + row) == (cell[0] - SX[q], cell[1] - SY[q]), (q, wi, wj)
                        assert (row, col) not in seen
                        seen.add((row, col))


def test_three_step_phase2_reads_where_phase1_wrote(src, f3):
    """Phase 2 slot (u, v) (window coordinates, u, v >= 1) takes population q from slot (u - sx_q,
    v - sy_q), a slot of the phase-1 window, at the position phase 1 wrote it (the kernel's su / sv),
    and writes over it: one reader and writer per position and population."""
    e = f3
    for q in range(4):
        seen = set()
        for v in range(1, 1 + e["kB3Y"]):
            for u in range(1, 1 + e["kB3X"]):
                su = _array(src, "void f3_tile(", "su", {"u": u, "v": v})
                sv = _array(src, "void f3_tile(", "sv", {"u": u, "v": v})
                assert (su[q], sv[q]) == (u - SX[q], v - SY[q]), (q, u, v)
                assert 0 <= su[q] < e["kW3X"] and 0 <= sv[q] < e["kW3Y"]
                assert (su[q], sv[q]) not in seen
                seen.add((su[q], sv[q]))


def test_three_step_phase3_reads_where_phase2_wrote(src, f3):
    """Phase 3 tile cell (lane, ty) is window slot (x, y) = (lane + 2, ty + 2); population q comes from
    inner slot (x - sx_q, y - sy_q), which phase 2 left at the position of its own source slot,
    (x - 2 sx_q, y - 2 sy_q): the kernel's px / py.  The edge pass that fills inner slots beyond a
    non-periodic side writes population q of slot (u, v) at (u - sx_q, v - sy_q) (its du / dv), where
    phase 3 looks.  The warps' rows cover the tile once."""
    e = f3
    for ty in range(e["kT3Y"]):
        for lane in range(e["kFTX"]):
            x, y = lane + 2, ty + 2
            px = _array(src, "void f3_tile(", "px", {"x": x, "y": y})
            py = _array(src, "void f3_tile(", "py", {"x": x, "y": y})
            for q in range(4):
                inner = (x - SX[q], y - SY[q])
                assert 1 <= inner[0] < 1 + e["kB3X"] and 1 <= inner[1] < 1 + e["kB3Y"], (q, lane, ty)
                assert (px[q], py[q]) == (inner[0] - SX[q], inner[1] - SY[q]), (q, lane, ty)
    body = src[src.index("void f3_tile("):]
    m = re.search(r"du\[4\] = \{([^}]*)\}, dv\[4\] = \{([^}]*)\}", body)
    assert m, "du / dv of f3_tile not found"
    du, dv = _int_exprs(m.group(1), {}), _int_exprs(m.group(2), {})
    assert du == [-s for s in SX] and dv == [-s for s in SY]
    nw = e["kT3T"] // 32
    rows = sorted(w + rep * nw for w in range(nw) for rep in range(e["kFTX"] * e["kT3Y"] // e["kT3T"]))
    assert rows == list(range(e["kT3Y"]))
