"""Host-side pieces of bench.py (no GPU): the roofline's DRAM traffic and
pipe utilisation are read from the committed ncu summaries of the kernel
and workload that the JSON line reports, and the simulated-time arithmetic."""
import math

import bench


def test_traffic_and_pipe_from_committed_profiles():
    # FP64 headline kernel and the FP32 window sweep on the bench workload
    for kernel in ("k_pair64", "k_pair32w"):
        traffic, src = bench.ncu_dram_bytes(kernel, "water512")
        assert src is not None and src.startswith("profiles/" + kernel + "_water512")
        assert 1e5 < traffic < 1e9  # bytes per launch: an L2-resident working set
        pipe = bench.ncu_pipe_pct(kernel, "water512")
        assert pipe is not None and 0.0 < pipe["pipe_pct"] <= 100.0
        assert pipe["source"] == src


def test_no_traffic_for_an_uncaptured_workload():
    # the electron workload has launch lists but no capture of these kernels:
    # the line must say null rather than borrow another workload's bytes
    assert bench.ncu_dram_bytes("k_pair64", "ion_electron") == (None, None)
    assert bench.ncu_pipe_pct("k_pair32w", "ion_electron") is None


def test_ns_per_day():
    # 1 ms per step of 0.25 fs: 86400 s/day * 1000 steps/s * 0.25e-6 ns
    assert math.isclose(bench.ns_per_day(1.0, 0.25), 21.6)
    assert math.isclose(bench.ns_per_day(0.5, 0.1), 17.28)
