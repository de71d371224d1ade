"""The in-place window of the two-steps-per-launch kernels, checked on the CPU.

The FP32 two-step kernel (forward) and the FP32 two-step adjoint sweep fetch, per population q,
one tensor-copy box of 36 x 18 cells whose origin is shifted by that population's velocity, and
write the first step's result for each window slot over the box positions it read.  That is
hazard-free only if (a) the position a slot reads for population q holds exactly the cell the
method pulls from (forward: x - c_q; adjoint: x + c_q), (b) no two slots read the same position of
a population's box, (c) every position lies inside its box, (d) the second step reads population q
of its source slot at that slot's position, and (e) every box starts on a 16-byte boundary
(x times 4 bytes).  The box origins, the position rule and the second step's source slots are read
from the kernel source, so the test follows the code.
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
