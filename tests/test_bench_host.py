"""Host logic of bench.py that needs no GPU: the source hash that gates the
DRAM traffic a bench line quotes from the committed ncu summary (only code
counts, not comments), and the lookup of that traffic by launch shape, number
of stream-K ranges and kind of sum."""
import os
import shutil

import pytest

import bench


def _tree(tmp_path):
    """A copy of the files the hash and the lookup read, under tmp_path."""
    src = os.path.join(bench.ROOT, "paper_2501_04456_gb300", "csrc")
    dst = tmp_path / "paper_2501_04456_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("allpairs_grouped.cu", "allpairs.cu", "npsim_internal.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    return dst


def _profile(tmp_path, h):
    (tmp_path / "profiles" / "allpairs_paper_scale250000.md").write_text(
        "dram bytes per charged-only launch, shape 21, 1216 ranges: 2.03e6\n"
        "dram bytes per full launch, shape 21, 1216 ranges: 5.62e6\n"
        f"source sha256[:16]: {h}\n")


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    dst = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash(2)
    with open(dst / "allpairs_grouped.cu", "a") as f:
        f.write("\n// a comment changes nothing\n/* nor does\n   a block comment */\n\n")
    assert bench.kernel_source_hash(2) == h0
    with open(dst / "npsim_internal.cuh", "a") as f:
        f.write("\nconstexpr int kAnotherConstant = 1;\n")
    assert bench.kernel_source_hash(2) != h0
    # the ungrouped kernels hash their own file
    assert bench.kernel_source_hash(0) != bench.kernel_source_hash(2)


def test_traffic_is_quoted_only_for_the_current_source(tmp_path, monkeypatch):
    dst = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    cfg = {"index": 21, "ranges": 1216, "packed": 2}
    _profile(tmp_path, bench.kernel_source_hash(2))
    assert bench._traffic_from_profile(cfg, full_sum=False) == pytest.approx(2.03e6)
    assert bench._traffic_from_profile(cfg, full_sum=True) == pytest.approx(5.62e6)
    # a launch shape or range count the capture does not cover
    assert bench._traffic_from_profile(dict(cfg, ranges=304), full_sum=False) is None
    assert bench._traffic_from_profile(dict(cfg, index=16), full_sum=False) is None
    # a kernel changed since the capture: nothing is quoted
    with open(dst / "allpairs_grouped.cu", "a") as f:
        f.write("\nconstexpr int kChanged = 2;\n")
    assert bench._traffic_from_profile(cfg, full_sum=False) is None
