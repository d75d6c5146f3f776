"""Host-side helpers of bench.py: the algorithmic byte counts behind the
roofline, the traffic lookup keyed by the kernel sources, the tile count of
the dependence build, and the oracle-rate extrapolation."""
import os

import numpy as np

import bench


def test_algorithmic_bytes_of_a_full_step():
    n, k = 20000, 32
    nt = -(-n // 128)
    state = 16 * n * k
    f32 = n * n * 4 + state + 2 * (2 * k * n * 4) + 2 * (max(k, 16) * n * 2)
    bf16 = n * n * 2 + state + 2 * (2 * k * n * 2)
    fp8 = n * n * 1 + state + 2 * (2 * k * n * 1) + 4 * nt * nt
    assert bench.alg_bytes_full_step(n, k, "f32", 0) == f32
    assert bench.alg_bytes_full_step(n, k, "bf16", 0) == bf16
    assert bench.alg_bytes_full_step(n, k, "fp8", 0) == fp8
    # RMSprop reads and writes its momentum too; ADMM's dual replaces G
    assert bench.alg_bytes_full_step(n, k, "f32", 1) == f32 + 8 * n * k
    assert bench.alg_bytes_full_step(n, k, "f32", 5) == f32


def test_traffic_lookup_follows_the_kernel_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "step_kernel_traffic.txt").write_text(
        "# comment\n"
        f"w_current {h} 123\n"
        "w_stale 0000000000000000 456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.measured_traffic("w_current") == 123.0
    assert bench.measured_traffic("w_stale") is None
    assert bench.measured_traffic("w_missing") is None


def test_committed_traffic_file_is_well_formed():
    p = os.path.join(bench.ROOT, "profiles", "step_kernel_traffic.txt")
    rows = [l.split() for l in open(p) if l.strip() and not l.startswith("#")]
    assert rows and all(len(r) == 3 and len(r[1]) == 16 and int(r[2]) > 0 for r in rows)
    for w, _, b in rows:
        kind, n, k, dt, method, _ = bench.WORKLOADS[w]
        ratio = int(b) / bench.alg_bytes_full_step(n, k, dt, method)
        assert 0.99 < ratio < 1.1, (w, ratio)


def test_dependence_tile_count_matches_enumeration():
    for n in (1, 127, 128, 300, 1000, 20000):
        nib, njb = (n + 127) // 128, (n + 255) // 256
        listed = sum(1 for jb in range(njb) for ib in range(nib) if 2 * jb + 1 >= ib)
        assert sum(min(nib, 2 * jb + 2) for jb in range(njb)) == listed


def test_oracle_row_rate_extrapolates_by_rows():
    rng = np.random.default_rng(0)
    S = rng.random((64, 4096))
    H = rng.random((4096, 8))
    r = bench.oracle_row_rate(S, H, np.arange(64), 4096, budget_s=0.2)
    assert r["kind"] == "oracle" and r["value"] > 0
    assert "x 64" in r["sample"]
