"""CPU checks of bench.py's host-side helpers: the DRAM traffic taken from a
committed ncu summary only while the kernel's sources still hash to the value
recorded there, the roofline fields derived from it, the peak source, and the
reference arm's silence on ranks other than 0."""
import io
import json
import os
from contextlib import redirect_stdout

import pytest

import bench


def test_dram_fields():
    assert bench.dram_fields(None, 1e-3, 6000.0) == {}
    d = bench.dram_fields(4.0e9, 2.0e-3, 5000.0)  # 4 GB in 2 ms = 2000 GB/s
    assert d["dram_achieved"] == pytest.approx(2000.0)
    assert d["dram_frac"] == pytest.approx(0.4)


def test_kernel_source_hash_is_stable_and_covers_every_source():
    for k in bench.KERNEL_SOURCES:
        h = bench.kernel_source_hash(k)
        assert len(h) == 16 and h == bench.kernel_source_hash(k)
        for name in bench.KERNEL_SOURCES[k]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2606_16959_gb300", "csrc", name))


def test_profiled_traffic_only_for_matching_sources(monkeypatch, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "qsweep_kernel_toy.md").write_text("# toy\n\nkernel_source_sha256: `0123456789abcdef`\n"
                                                "dram_bytes_per_launch: `4295463680`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "0123456789abcdef")
    assert bench.profiled_traffic("toy", "qsweep_kernel") == 4295463680.0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "fedcba9876543210")
    assert bench.profiled_traffic("toy", "qsweep_kernel") is None  # sources changed since the capture
    assert bench.profiled_traffic("other", "qsweep_kernel") is None  # no summary
    assert bench.profiled_traffic("toy", "no_such_kernel") is None


def test_committed_summaries_parse():
    """Every committed summary that records traffic gives its hash and a
    positive byte count in the form profiled_traffic reads."""
    d = os.path.join(bench.ROOT, "profiles")
    for name in sorted(os.listdir(d)):
        text = open(os.path.join(d, name)).read()
        if "dram_bytes_per_launch" not in text:
            continue
        vals = {}
        for line in text.splitlines():
            if line.strip().startswith(("kernel_source_sha256", "dram_bytes_per_launch")):
                k, v = line.strip().strip("`").split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
        assert len(vals["kernel_source_sha256"]) == 16, name
        assert float(vals["dram_bytes_per_launch"]) > 0, name


def test_peaks_read_the_measured_file():
    hbm, kind = bench.peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")) as fh:
            assert hbm == float(json.load(fh)["hbm_gbs"]) and kind == "measured"
    else:
        assert (hbm, kind) == (6800.0, "fallback")


def test_reference_arm_silent_on_other_ranks(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.run_reference(None) is None
    assert out.getvalue() == ""
