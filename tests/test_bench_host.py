"""Host-side arithmetic of the benchmark's JSON line (no GPU): the union of launch intervals,
the roofline record built from them, the DRAM-traffic record that is reported only while the
step kernel's sources are the ones it was captured from, the batch-means standard error and
the snapshot copy count of the end-to-end arm."""
import math

import numpy as np
import pytest

import bench


def test_union_of_launch_intervals():
    assert bench.union_ms(np.zeros((0, 2))) == 0.0
    iv = np.array([[5.0, 6.0], [0.0, 2.0], [1.0, 3.0], [1.5, 2.5]])
    assert bench.union_ms(iv) == pytest.approx(4.0)          # [0, 3] and [5, 6]
    assert bench.union_ms(np.array([[0.0, 10.0], [2.0, 3.0]])) == pytest.approx(10.0)


def test_roofline_record_arithmetic():
    """Two overlapping launches (two streams): achieved bandwidth over the union of their
    intervals, per-launch figures over the launch count, traffic scaled per launch."""
    iv = np.array([[0.0, 10.0], [5.0, 15.0]])
    l1 = {1: 40000.0, 2: 42000.0}
    tr = {"dram_bytes_per_particle_step": 0.5, "source": "rec", "l1": {"wavefronts_per_warp_step": 377.0}}
    r = bench.roofline_record(iv, 1e9, 1152, l1, None, tr)
    assert r["bound"] == "l1" and r["unit"] == "GB/s"
    assert r["kernel_ms_union"] == pytest.approx(15.0)
    assert r["achieved"] == pytest.approx(1e9 * 1152 / 0.015 / 1e9)
    assert r["peak"] == 42000.0
    assert r["frac"] == pytest.approx(r["achieved"] / 42000.0)
    assert r["traffic"] == pytest.approx(0.5 * 1e9 / 2)
    assert r["alg_bytes_per_launch"] == pytest.approx(1152e9 / 2)
    assert r["kernel_launches"] == 2
    assert r["kernel_ms_total"] == pytest.approx(20.0) and r["kernel_ms_mean_launch"] == pytest.approx(10.0)
    assert r["l1_wavefronts"]["wavefronts_per_warp_step"] == 377.0
    none = bench.roofline_record(iv, 1e9, 1152, l1, None, None)
    assert none["traffic"] is None and none["l1_wavefronts"] is None


def test_traffic_record_follows_the_kernel_sources(monkeypatch):
    """The committed ncu record is reported while the step kernel's sources hash to the value it
    was captured with, for each storage form it holds; any other hash (a changed kernel) or
    another record layout leaves it unreported."""
    import json
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.load(f)
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: rec["sources_sha256"])
    for dt in rec["by_dtype"]:
        t = bench.measured_traffic("cell", dt)
        assert t is not None, dt
        assert 0.0 < t["dram_bytes_per_particle_step"] < 10.0
        assert t["l1"]["wavefronts_per_warp_step"] >= t["l1"]["floor"]
    assert bench.measured_traffic("cell", "f64") is None
    assert bench.measured_traffic("pair") is None
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0" * 64)
    assert bench.measured_traffic("cell") is None


def test_batch_means_standard_error():
    """sqrt(32 var(class sums)) for the sum over particles: exact on a small case, and for
    independent draws close to sqrt(N) times their standard deviation."""
    x = np.arange(64, dtype=float)
    s = np.array([i + (i + 32) for i in range(32)], dtype=float)
    assert bench.batch_sigma(x) == pytest.approx(math.sqrt(32 * s.var(ddof=1)))
    rng = np.random.default_rng(0)
    y = rng.normal(0.0, 2.0, size=320_000)
    assert bench.batch_sigma(y) == pytest.approx(math.sqrt(len(y)) * 2.0, rel=0.35)


def test_ring_upload_count():
    """The copy count behind the end-to-end line's h2d_bytes_per_step: with one slot per
    snapshot of a periodic sequence every snapshot crosses once per step however many periods
    the run spans; with a smaller ring every unwrapped snapshot the run reaches crosses once
    (time only moves forward); a non-periodic sequence is copied once, its frozen tail
    included."""
    hourly_4d = [(i * 360, (i + 1) * 360, i) for i in range(96)]          # 4 days, 24 snapshots
    assert bench.ring_uploads(hourly_4d, 24, 24, True) == 24
    runs = [(i * 60, (i + 1) * 60, i) for i in range(14)]                  # 2.3 periods of 6
    assert bench.ring_uploads(runs, 6, 6, True) == 6
    for R in (2, 3, 4):
        assert bench.ring_uploads(runs, R, 6, True) == 15                  # snapshots 0 .. 14
    frozen = [(i * 60, (i + 1) * 60, i) for i in range(5)] + [(300, 800, -1 - 5)]
    for R in (2, 3, 6):
        assert bench.ring_uploads(frozen, R, 6, False) == 6
