"""bench.py helpers on the CPU: the committed ncu traffic figure is used only for the kernel
source it was captured from (comments and blank lines aside)."""

import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = os.path.join("paper_1705_04384_gb300", "csrc", "kernels_fd64.cu")


def _tree(tmp_path, edit=None):
    dst = tmp_path / SRC
    dst.parent.mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, SRC), dst)
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "fd_fold_mma_3d_ne64.md"),
                tmp_path / "profiles" / "fd_fold_mma_3d_ne64.md")
    if edit:
        dst.write_text(edit(dst.read_text()))
    return str(tmp_path)


def test_hash_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path))
    h0 = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "a", lambda s: "// a note\n\n" + s.replace(
        "namespace iga {", "namespace iga {  // trailing comment\n\n")))
    assert bench.kernel_source_hash() == h0
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "b", lambda s: s.replace(
        "kMmaWps = 2", "kMmaWps = 1")))
    assert bench.kernel_source_hash() != h0


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "b", lambda s: s.replace(
        "kMmaWps = 2", "kMmaWps = 1")))
    assert bench.committed_traffic("fd_fold_mma_3d_ne64.md") is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "missing"))
    assert bench.committed_traffic("fd_fold_mma_3d_ne64.md") is None


def test_traffic_of_an_unchanged_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path))
    val = bench.committed_traffic("fd_fold_mma_3d_ne64.md")
    if val is not None:  # the committed capture matches the current source
        assert val > 0


def test_algorithmic_counts():
    # folded FD mode product at n = 65 (3D): the committed summary's 17.99 MFLOP per launch
    assert abs(bench.fold_flops_per_launch(65, 3) - 17.99e6) < 0.01e6
    # dense equivalent is twice as large up to the odd middle entry
    n = 130
    assert abs(bench.fold_flops_per_launch(n, 3) - n ** 4) / n ** 4 < 1e-12
    # operator on the extruded annulus, p = 3 (W = 4): 9 band passes of 2W + 2 per term
    assert bench.operator_flops_per_dof(4) == 2 * 4 * 9 + 8


def test_percentile():
    assert bench.percentile([3.0, 1.0, 2.0], 50) == 2.0
