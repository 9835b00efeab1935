"""Host logic of bench.py that needs no GPU: step statistics, the FFT flop
model behind the FP32 roofline, the traffic table's source key, and the
number of eager steps with per-stage kernel events (one per PROFILE_EVERY
timed steps)."""
import math

import bench


def test_step_stats_split_and_quantiles():
    steps = [0.70, 0.71, 0.69, 0.80, 0.70, 0.70, 0.72, 0.79]
    st = bench.step_stats(steps, [0.76, 0.78])
    assert st["with_kernel_events_median"] in (0.76, 0.78)
    assert st["p10"] <= st["median"] <= st["p90"]
    assert min(steps) <= st["p10"] and st["p90"] <= max(steps)
    empty = bench.step_stats([0.5], [])
    assert empty["median"] == 0.5 and empty["with_kernel_events_median"] is None


def test_fft_flop_model_by_hand():
    """5 N log2 N per complex FFT of length N (half for a real row), both
    column transforms plus the kernel product, per forward + adjoint step."""
    piece = dict(Ptheta=16, Prho=32, Ntheta=10, k1max=5, k2max=3)
    fl = bench.fft_flops_per_step([piece])
    col = 4 * (2 * 5 * 16 * 4 + 6 * 11)          # 4 columns: forward + inverse FFT of 16, 11 products
    rows = 10 * 0.5 * 5 * 32 * 5                  # 10 real rows of 32
    assert math.isclose(fl["k_colconv"], 2 * col)
    assert math.isclose(fl["k_rows_r2c"], rows) and math.isclose(fl["k_band_rows"], rows)
    assert math.isclose(fl["k_rows_c2r"], 2 * rows)
    two = bench.fft_flops_per_step([piece, piece])
    assert all(math.isclose(two[k], 2 * fl[k]) for k in fl)


def test_traffic_table_lookup_follows_the_source_digest(monkeypatch):
    digest = bench.kernel_source_digest()
    assert len(digest) == 16 and int(digest, 16) >= 0
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "k_test", (digest, 1.5e6))
    assert bench.measured_traffic("k_test") == 1.5e6
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "k_test", ("0" * 16, 1.5e6))
    assert bench.measured_traffic("k_test") is None           # stale: no traffic figure
    assert bench.measured_traffic("k_unknown") is None


def test_profiled_steps_are_a_bounded_share():
    """Eager steps with per-kernel events after the timed ones: one per
    PROFILE_EVERY timed steps, at least one."""
    for K in (1, 2, 3, 4, 10, 20):
        n = bench.profiled_steps(K)
        assert 1 <= n <= max(1, K // bench.PROFILE_EVERY)
    assert bench.profiled_steps(20) == 5
