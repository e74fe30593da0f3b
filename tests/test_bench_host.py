"""Host-side pieces of bench.py that shape the reported line: the traffic
lookup keyed by the kernel sources, the roofline extras, the interval
statistics, the kernel naming of the two-array, streaming and wavefront
modes and the replica throughput."""
import math

import pytest

import bench


def test_traffic_lookup_follows_the_kernel_sources():
    """A summary's traffic counts only while its recorded source hash is that
    of the sources named; any other source set (a changed kernel) gives none."""
    import re
    name = "k_step_rows2_async_f32r_grf256.md"
    text = open(bench.os.path.join(bench.ROOT, "profiles", name)).read()
    recorded = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text).group(1)
    tb = int(re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text).group(1))
    assert bench.profile_traffic(name) == (tb if recorded == bench.kernel_sha() else None)
    assert bench.profile_traffic(name, ["paper_2304_11165_b300/csrc/sbg_reduce.cu"]) is None
    assert bench.profile_traffic("no_such_summary.md") is None


def test_roofline_extras():
    r = {"bound": "hbm", "achieved": 2600.0, "peak": 6500.0, "traffic": 80e6, "avg_launch_us": 25.0}
    bench.roofline_extras(r)
    assert r["frac_nominal"] == pytest.approx(2600.0 / bench.NOMINAL_HBM_GBS)
    assert r["dram_gbs_from_traffic"] == pytest.approx(80e6 / 25e-6 / 1e9)
    assert r["dram_frac_from_traffic"] == pytest.approx(3200.0 / 6500.0)
    r2 = {"bound": "hbm", "achieved": 10.0, "peak": 6500.0, "traffic": None, "avg_launch_us": 1.0}
    bench.roofline_extras(r2)
    assert "dram_gbs_from_traffic" not in r2 and "frac_nominal" in r2
    r3 = {"bound": "alu", "achieved": 1.0}
    assert bench.roofline_extras(dict(r3)) == r3


def test_interval_statistics():
    s = bench.interval_stats([7.0, 7.2, 6.8, 7.0], 256)
    assert s["n_intervals"] == 4
    assert s["mean_us_per_rd_step"] == pytest.approx(7.0 / 256 * 1e3)
    sd = math.sqrt(((0.2 / 256) ** 2 * 2) / 3) * 1e3
    assert s["stderr_us"] == pytest.approx(sd / 2)
    assert bench.interval_stats([5.0], 10)["stderr_us"] is None
    assert bench.interval_stats([], 10) is None


def test_kernel_names_of_the_two_array_modes():
    assert bench.two_array_kernel("async") == "k_step_rows2"
    assert bench.two_array_kernel("pipelined") == "k_step_pipe"
    assert bench.two_array_kernel("prefetch") == "k_step_pipe"
    assert bench.two_array_kernel("plain") == "k_step"
    assert bench.two_array_kernel("stream") == "k_step_stream_inh"


def test_streaming_and_wavefront_kernels_are_named_and_keyed():
    """The reactive bench names the streaming kernel (or the wavefront kernel,
    which runs 2 or 4 steps per launch) and keys its ncu summary to the hash of
    that kernel's own sources."""
    assert bench.step_kernel_name(2, "stream") == "k_step_stream"
    assert bench.step_kernel_name(2, "wave") == bench.step_kernel_name(2, "wave4") == "k_step_wave"
    assert bench.step_kernel_name(2, "async") == "k_step_rows2"
    assert bench.step_kernel_name(1, "plain") == "k_step"
    assert [bench.steps_per_launch(v) for v in ("stream", "wave", "wave4", "async")] == [1, 2, 4, 1]
    for k in ("k_step_stream", "k_step_stream_inh", "k_step_stream_x2"):
        assert bench.step_kernel_sources(k) == bench.STREAM_SOURCES
    assert bench.step_kernel_sources("k_step_wave") == bench.WAVE_SOURCES
    assert bench.step_kernel_sources("k_step_rows2") == bench.KERNEL_SOURCES


def test_replica_throughput_counts_every_rank():
    assert bench.replica_throughput(1e9, 4, 2000.0) == pytest.approx(2e9)
