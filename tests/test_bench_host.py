"""Host-side bookkeeping of bench.py's roofline line: the ncu traffic of a
kernel is used only while the sources that kernel is compiled from are the
ones the capture was taken on."""
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and the traffic summary, with bench.ROOT
    pointing at it."""
    import bench
    for rel in ("paper_2009_12623_gb300/csrc", "include", "profiles"):
        shutil.copytree(os.path.join(ROOT, rel), tmp_path / rel,
                        ignore=shutil.ignore_patterns("*.o", "*.so", "__pycache__"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path, bench


def _touch(path):
    with open(path, "a") as f:
        f.write("\n// edited\n")


def test_traffic_scaled_by_cells_while_sources_match(tree):
    root, bench = tree
    d = json.load(open(root / "profiles" / "ncu_traffic.json"))
    for k in ("stencil_forward", "stencil_adjoint", "zfp_encode", "zfp_decode"):
        e = d[k]
        assert bench.measured_traffic(k, e["cells"]) == round(e["dram_bytes_per_launch"])
        assert bench.measured_traffic(k, 2 * e["cells"]) == round(2 * e["dram_bytes_per_launch"])


def test_each_kernel_hashes_its_own_sources(tree):
    root, bench = tree
    csrc = root / "paper_2009_12623_gb300" / "csrc"
    before = {k: bench.source_hash(k) for k in ("stencil_forward", "zfp_encode")}
    _touch(csrc / "codec_block.cuh")  # the codec's header: the stencil does not include it
    assert bench.source_hash("stencil_forward") == before["stencil_forward"]
    assert bench.source_hash("zfp_encode") != before["zfp_encode"]
    _touch(csrc / "common.cuh")  # included by both
    assert bench.source_hash("stencil_forward") != before["stencil_forward"]
    cells = json.load(open(root / "profiles" / "ncu_traffic.json"))["stencil_forward"]["cells"]
    assert bench.measured_traffic("stencil_forward", cells) is None
    assert bench.measured_traffic("zfp_decode", cells) is None
