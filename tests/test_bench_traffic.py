"""bench.py's recorded DRAM traffic: a figure from a committed ncu summary is
used only while the kernel's source file is byte-for-byte the one profiled
(its SHA-256 in the summary); otherwise, or when the summary is missing or
malformed, the roofline's traffic is null. Checked on CPU in a scratch tree."""

import hashlib
import os

import bench


def _tree(tmp_path, src=b"__global__ void k() {}\n"):
    csrc = tmp_path / "paper_2204_04898_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "format.cu").write_bytes(src)
    (tmp_path / "profiles").mkdir()
    return hashlib.sha256(src).hexdigest()


def _summary(tmp_path, sha, traffic="7172100953"):
    (tmp_path / "profiles" / "partition_very_large_log.md").write_text(
        "# partition\n\n- source_sha256: `%s`\n- dram_bytes_per_launch: %s\n" % (sha, traffic))


def test_current_source_gives_the_figure(tmp_path, monkeypatch):
    sha = _tree(tmp_path)
    _summary(tmp_path, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("partition", "very_large_log") == 7172100953.0


def test_changed_source_gives_null(tmp_path, monkeypatch):
    sha = _tree(tmp_path)
    _summary(tmp_path, sha)
    (tmp_path / "paper_2204_04898_b300" / "csrc" / "format.cu").write_bytes(b"__global__ void k() { }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("partition", "very_large_log") is None


def test_missing_or_malformed_gives_null(tmp_path, monkeypatch):
    sha = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("partition", "very_large_log") is None      # no summary
    assert bench.recorded_traffic("stats", "very_large_log") is None          # no source recorded
    _summary(tmp_path, sha, traffic="n/a")
    assert bench.recorded_traffic("partition", "very_large_log") is None


def test_committed_summaries_name_existing_sources():
    """Every committed summary that records a traffic figure belongs to a
    kernel whose source file exists."""
    prof = os.path.join(bench.ROOT, "profiles")
    for name in os.listdir(prof):
        text = open(os.path.join(prof, name)).read()
        if "dram_bytes_per_launch" not in text:
            continue
        kernel = next((k for k in bench.KERNEL_SOURCE if name.startswith(k + "_")), None)
        assert kernel is not None, name
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2204_04898_b300", "csrc",
                                           bench.KERNEL_SOURCE[kernel])), name
