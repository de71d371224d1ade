"""The scope of the hash that ties the bench's DRAM-traffic record to the three-step kernel.

bench.py reports `traffic` for the three-step kernel from a committed ncu record only while the hash of
the code that kernel's launches depend on matches the record.  The hash must change with any edit to
that code (the shared device helpers, the FP32 kernel file up to the end of the three-step kernel, the
three-step launcher) and must not change with edits elsewhere in the file (the scalar and adjoint
kernels after it, other launchers).  Checked on copies of the sources with planted edits.
"""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join("paper_1504_07034_gb300", "csrc")
SCALAR = b"// ---------------------------------------------------------------- scalar D2Q4, two steps per launch"
LAUNCHER = b"// The distance of the three-step kernel's L2 prefetch"
AFTER_LAUNCHER = b"cudaError_t launch_step2_f32("


@pytest.fixture
def tree(tmp_path, monkeypatch):
    os.makedirs(tmp_path / CSRC)
    for name in ("lbrs_kernels.cuh", "lbrs_kernels_f32.cu"):
        shutil.copy(os.path.join(ROOT, CSRC, name), tmp_path / CSRC / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _edit(tree, name, at, before=True):
    """Insert a comment line just before (or just after) the first occurrence of marker `at`."""
    path = tree / CSRC / name
    text = path.read_bytes()
    i = text.find(at)
    assert i >= 0, at
    if not before:
        i = text.find(b"\n", i) + 1
    path.write_bytes(text[:i] + b"// planted edit\n" + text[i:])


def test_markers_present_in_the_sources():
    text = open(os.path.join(ROOT, CSRC, "lbrs_kernels_f32.cu"), "rb").read()
    pos = [text.find(m) for m in (b"step2d_f32_fused3_kernel(", SCALAR, LAUNCHER, AFTER_LAUNCHER)]
    assert min(pos) >= 0
    assert pos[0] < pos[1], "the three-step kernel must come before the scalar section"
    assert pos[2] < pos[3]


@pytest.mark.parametrize("name, at, before, changes", [
    ("lbrs_kernels_f32.cu", b"step2d_f32_fused3_kernel(", True, True),     # inside the three-step kernel's span
    ("lbrs_kernels_f32.cu", SCALAR, True, True),                           # last line of the span
    ("lbrs_kernels.cuh", b"rcp_f32", True, True),                          # a shared device helper
    ("lbrs_kernels_f32.cu", LAUNCHER, False, True),                        # the three-step launcher
    ("lbrs_kernels_f32.cu", SCALAR, False, False),                         # the scalar kernel
    ("lbrs_kernels_f32.cu", b"adj_fused2_u_kernel(", True, False),         # the adjoint sweep
    ("lbrs_kernels_f32.cu", AFTER_LAUNCHER, False, False),                 # the two-step launcher
])
def test_hash_follows_the_three_step_code_only(tree, name, at, before, changes):
    h0 = bench.kernel_source_sha()
    _edit(tree, name, at, before)
    assert (bench.kernel_source_sha() != h0) == changes


def test_record_is_dropped_when_the_hash_differs(tree):
    rec = json.load(open(os.path.join(ROOT, "profiles", "step2d_f32_fused3_traffic.json")))
    assert rec["cells"] > 0 and rec["dram_bytes_per_launch"] > 0
    os.makedirs(tree / "profiles")
    rec["source_sha"] = bench.kernel_source_sha()
    (tree / "profiles" / "step2d_f32_fused3_traffic.json").write_text(json.dumps(rec))
    assert bench.measured_traffic(2 * rec["cells"]) == pytest.approx(2 * rec["dram_bytes_per_launch"])
    _edit(tree, "lbrs_kernels_f32.cu", b"step2d_f32_fused3_kernel(")
    assert bench.measured_traffic(rec["cells"]) is None
