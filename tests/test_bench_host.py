"""Host-side bookkeeping of bench.py: the DRAM traffic it reports for the
dominant kernel comes from the committed ncu summary only while the CUDA
sources are the ones that summary was captured on; any change makes it null."""
import os
import shutil

import bench


def _copy_tree(tmp_path):
    """A copy of the kernel sources and the traffic table in which bench's
    ROOT-relative paths can be pointed at."""
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2509_07021_gb300", "csrc"),
                    root / "paper_2509_07021_gb300" / "csrc")
    (root / "profiles").mkdir()
    shutil.copy(bench.TRAFFIC_TABLE, root / "profiles" / "dram_traffic_1m_1080p.md")
    return root


def _point_bench_at(monkeypatch, root):
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", str(root / "profiles" / "dram_traffic_1m_1080p.md"))


def test_committed_table_matches_committed_sources():
    # the committed summary names the digest of the committed CUDA sources
    text = open(bench.TRAFFIC_TABLE).read()
    assert bench.kernel_source_digest() in text
    for stage in ("blend_bwd", "blend_fwd", "preprocess", "preprocess_bwd", "duplicate"):
        v = bench.recorded_traffic(stage)
        assert v is not None and v > 1e6, stage


def test_any_source_change_voids_the_traffic(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    _point_bench_at(monkeypatch, root)
    assert bench.recorded_traffic("blend_bwd") is not None
    blend = root / "paper_2509_07021_gb300" / "csrc" / "sg_blend.cu"
    blend.write_text(blend.read_text() + "\n// edited\n")
    assert bench.recorded_traffic("blend_bwd") is None


def test_unknown_stage_and_missing_table(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    _point_bench_at(monkeypatch, root)
    assert bench.recorded_traffic("no_such_stage") is None
    os.remove(root / "profiles" / "dram_traffic_1m_1080p.md")
    assert bench.recorded_traffic("blend_bwd") is None
