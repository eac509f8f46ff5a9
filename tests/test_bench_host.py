"""Host-side logic of the benchmark (no GPU): the DRAM traffic it reports
beside the splat's roofline comes from a committed ncu summary only while
the kernel's sources hash to the ones captured, and a comment edit does not
orphan the summary."""
import os

import pytest

import bench


def _fake_tree(tmp_path, src: str):
    root = tmp_path / "repo"
    csrc = root / "paper_2601_19901_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src)
    (root / "profiles").mkdir()
    return root


def _profile(root, digest: str, rd="200.5", wr="40.25"):
    (root / "profiles" / "k.md").write_text(
        "# k\n\nKernel sources at capture sha256: %s\n\n| metric | value |\n|---|---|\n"
        "| DRAM read (`dram__bytes_read.sum`) | %s Mbyte |\n| DRAM write (`dram__bytes_write.sum`) | %s Mbyte |\n"
        % (digest, rd, wr))


def test_traffic_only_while_the_sources_match(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path, "__global__ void k() { int x = 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    d = bench.source_digest(["k.cu"])
    _profile(root, d)
    assert bench.profiled_traffic("k.md", ["k.cu"]) == pytest.approx(240.75e6)
    # comments and blank space do not change the digest
    (root / "paper_2601_19901_gb300" / "csrc" / "k.cu").write_text(
        "// a note\n__global__ void k() {\n  int x = 1;   /* same */\n}\n")
    assert bench.source_digest(["k.cu"]) == d
    assert bench.profiled_traffic("k.md", ["k.cu"]) == pytest.approx(240.75e6)
    # a code change does
    (root / "paper_2601_19901_gb300" / "csrc" / "k.cu").write_text("__global__ void k() { int x = 2; }\n")
    assert bench.source_digest(["k.cu"]) != d
    assert bench.profiled_traffic("k.md", ["k.cu"]) is None


def test_missing_profile_or_counters_give_no_traffic(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path, "__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic("k.md", ["k.cu"]) is None
    (root / "profiles" / "k.md").write_text("sha256: %s\n" % bench.source_digest(["k.cu"]))
    assert bench.profiled_traffic("k.md", ["k.cu"]) is None


def test_the_committed_splat_summary_parses():
    text = open(os.path.join(bench.ROOT, "profiles", "k_splat_paper_frame.md")).read()
    assert "sha256:" in text and "dram__bytes_read.sum" in text and "dram__bytes_write.sum" in text


def test_reduced_scene_only_for_the_paper_shaped_configs():
    with pytest.raises(SystemExit):
        bench.workload("pbr", 40)
