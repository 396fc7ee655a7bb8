"""The benchmark's host-side arithmetic (no GPU): the algorithmic counts its
roofline divides by, checked against hand counts of the bench workloads, the
chain's byte count, and the parsing of the committed ncu summaries."""
import os

import bench


def test_fp32_flop_counts():
    # four Gaussian peaks in 8-D: map 4 D + peaks K (3 D + 2) + moments 10
    assert bench.flops_per_sample(8, 4) == 32 + 4 * 26 + 10 == 146
    # the 20-D ball: map 4 D + test 2 D + 1 + moments 10
    assert bench.ball_flops_per_sample(20) == 80 + 41 + 10 == 131


def test_lane_operation_counts():
    # Philox 60 per call (6 per round, 10 rounds), ceil(D/4) calls
    assert bench.ops_per_sample(8, 4) == 2 * 60 + 7 * 8 + 4 * 19 + 10 + 16 == 278
    assert bench.ops_per_sample(20, 1, ball=True) == 5 * 60 + 7 * 20 + 42 + 10 + 40 == 532


def test_chain_bytes():
    bench._LAST_CHAIN_MS[0] = 0.5
    v = bench._chain_view(1 << 20, 20, 1000, 6767.4)
    assert v["bytes_per_iteration"] == 68 * (1 << 20) + 12 * 20 * 1000
    assert abs(v["achieved_gbs"] - v["bytes_per_iteration"] / 0.5e-3 / 1e9) < 1e-6
    assert abs(v["frac"] - v["achieved_gbs"] / 6767.4) < 1e-12
    bench._LAST_CHAIN_MS[0] = 0.0
    assert "frac" not in bench._chain_view(1 << 20, 20, 1000, 6767.4)


def test_committed_profiles_parse():
    """Each committed sampling-kernel summary names the source it was taken on
    and carries the DRAM bytes and the pipe percentages the bench line reads."""
    for (workload, n_ev), name in bench.PROFILE_FILES.items():
        text = open(os.path.join(bench.ROOT, "profiles", name)).read()
        keys = dict(line.split(":", 1) for line in text.splitlines()[:8] if ":" in line)
        assert len(keys["kernel_source_sha1"].strip()) == 40
        assert int(keys["profiled_samples"]) > 0 and int(keys["dram_bytes_per_launch"]) > 0
        for k in bench.PIPE_KEYS:
            assert 0.0 < float(keys[k + "_pct_elapsed"].split()[0]) < 100.0
        fig = bench.profile_figures(workload, keys["kernel_source_sha1"].strip(), n_ev)
        assert fig is not None and fig["traffic_per_sample"] > 0
        assert bench.profile_figures(workload, "0" * 40, n_ev) is None
        assert bench.profile_figures(workload, keys["kernel_source_sha1"].strip(), 12345) is None
