"""Host-side bookkeeping of bench.py: the DRAM traffic it reports for the
dominant kernel is the recorded ncu figure only while the CUDA sources are the
ones the capture was taken on; any change makes it null."""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2509_07021_gb300", "csrc"),
                    root / "paper_2509_07021_gb300" / "csrc")
    return root


def test_recorded_traffic_needs_the_captured_sources(tmp_path):
    root = _copy_sources(tmp_path)
    table = {"sources": bench.kernel_source_digest(str(root)), "bytes": {"blend_bwd": 1.25e8}}
    assert bench.recorded_traffic("blend_bwd", table, str(root)) == 1.25e8
    assert bench.recorded_traffic("no_such_stage", table, str(root)) is None
    blend = root / "paper_2509_07021_gb300" / "csrc" / "sg_blend.cu"
    blend.write_text(blend.read_text() + "\n// edited\n")
    assert bench.recorded_traffic("blend_bwd", table, str(root)) is None


def test_committed_record_is_current_or_null():
    """The committed record either names the committed sources or yields null."""
    t = bench.RECORDED_TRAFFIC
    for stage in ("blend_bwd", "blend_fwd", "preprocess"):
        v = bench.recorded_traffic(stage)
        if t["sources"] == bench.kernel_source_digest():
            assert v is None or v > 1e6
        else:
            assert v is None


def test_step_statistics():
    st = bench.step_stats([2.0, 1.0, 4.0, 3.0])
    assert st["median"] == 2.5 and st["min"] == 1.0 and st["max"] == 4.0 and st["mean"] == 2.5
