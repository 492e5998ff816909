"""CPU tests of bench.py's helpers: the roofline's DRAM traffic is taken from an
ncu summary only while that summary's digest matches the stochastic step's
sources, and the measured peaks load from their file."""
import bench


def _summary(tmp_path, digest, nbytes=123456):
    p = tmp_path / "k.md"
    p.write_text(f"# summary\n\n- `dram_bytes_per_launch: {nbytes}`\n- `sources_sha256: {digest}`\n")
    return str(p)


def test_traffic_read_while_sources_match(tmp_path):
    assert bench.profiled_traffic(_summary(tmp_path, bench.kernel_sources_digest())) == 123456.0


def test_traffic_dropped_when_sources_changed(tmp_path):
    assert bench.profiled_traffic(_summary(tmp_path, "0" * 64)) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md")) is None


def test_digest_covers_the_stochastic_step_sources_only():
    assert "ssa.cu" in bench.SSA_SOURCES and "ssa_device.cuh" in bench.SSA_SOURCES
    assert not any(s.startswith("general") or s.startswith("events") for s in bench.SSA_SOURCES)
    assert len(bench.kernel_sources_digest()) == 64


def test_measured_peaks_is_a_mapping():
    assert isinstance(bench.measured_peaks(), dict)


class _W:
    model, N, nc, T = 3, 37_000, 6, 1460


def test_roofline_fraction_follows_from_its_inputs():
    # frac = (40 FP64 lane-ops per draw x (transitions + node-days) / launches)
    #        / average launch time of the stochastic step timed alone / measured peak
    transitions, T, peak = 109_901_254, 1460, 5.0e11
    alone = {"ms_per_launch": 0.0146, "launches": T, "transitions": transitions, "node_days": _W.N * T}
    r = bench.ssa_roofline(_W, 1, alone, peak, ms_per_step=28.9, hbm_peak=6762.6)
    avg_s = 0.0146 / 1000
    ops = 40 * (transitions + _W.N * T) / T
    assert abs(r["frac"] - ops / avg_s / peak) < 1e-12
    assert abs(r["achieved"] * 1e9 - ops / avg_s) < 1e-3
    assert r["fits_in_ms_per_step"]
    assert abs(r["hbm"]["achieved"] - 64 * _W.N / avg_s / 1e9) < 1e-9
    spec = (15 * transitions + 34 * _W.N * T) / T / avg_s / peak
    assert abs(r["frac_spec_count"] - spec) < 1e-12
    r2 = bench.ssa_roofline(_W, 1, alone, peak, ms_per_step=10.0, hbm_peak=6762.6)
    assert not r2["fits_in_ms_per_step"]
