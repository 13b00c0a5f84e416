"""bench.py's host-side helpers, on the CPU: the prefilter sample-set choice,
the host-memory probe that gates the batch form's end-to-end run, and the
lookup of DRAM bytes from the committed ncu summaries (null when the kernel's
source changed since the capture)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_prefilter_sample_choice_is_balanced_and_seeded():
    import paper_1810_08860_gb300 as lfm

    S, seed, balance = bench.pick_prefilter_samples(lfm, 32)
    assert S.dtype == np.float32 and S.shape == (32, 4)
    assert balance > 0.6
    assert np.array_equal(S, lfm.prefilter_samples(32, seed))
    S64 = S.astype(np.float64)
    w = (1 - np.sqrt(S64[:, 0])) * np.sinc(S64[:, 2]) * np.sinc(S64[:, 2] / 2) * np.sinc(S64[:, 3]) * np.sinc(S64[:, 3] / 2)
    assert abs(w.sum() / np.abs(w).sum() - balance) < 1e-9


def test_host_memory_probe():
    avail = bench.host_memory_available()
    assert avail > 0
    with open("/proc/meminfo") as fh:
        total = int(next(l for l in fh if l.startswith("MemTotal:")).split()[1]) * 1024
    assert avail <= total


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    assert bench.ncu_traffic("no_such_profile") is None
    # a summary gives its bytes only while its hash matches the source's
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "fresh.txt").write_text("kernel_source_sha: 1111111111111111\ndram_bytes_per_launch: 123\n")
    (prof / "stale.txt").write_text("kernel_source_sha: 0000000000000000\ndram_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files=bench.RASTER_SOURCES: "1111111111111111")
    assert bench.ncu_traffic("fresh") == 123.0
    assert bench.ncu_traffic("stale") is None
