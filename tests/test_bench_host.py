"""Host-side arithmetic of the benchmark line (no GPU): roofline denominators from the measured
peaks, the committed DRAM traffic figure, and the workload recipes the bench times."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _stats(ms=20.0):
    return {"toeplitz_ms": ms, "toeplitz_flops": 0.0, "toeplitz_bytes": 0.0}


@pytest.mark.parametrize("prec,products", [("bf16x3", 6), ("bf16x2", 3), ("tf32x3", 6)])
def test_tensor_roofline_uses_measured_bf16_peak(bench, prec, products):
    """The split precisions are measured against the burst BF16 rate of the peaks file (the
    products are timed in sub-second regions) divided by the tensor-core products each useful
    product costs; frac = achieved / peak."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16 = float(json.load(open(path))["bf16_tflops"]) if os.path.exists(path) else 1900.0
    r = bench.roofline(prec, 150.0, 7.0e8, 10, _stats(30.0), 60.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(bf16 / products)
    assert r["frac"] == pytest.approx(150.0 / (bf16 / products))
    assert r["avg_launch_ms"] == pytest.approx(3.0) and r["share_of_step"] == pytest.approx(0.5)
    assert r["traffic"] == 7.0e8 and r["launches"] == 10


@pytest.mark.parametrize("prec", ["fft32", "fp32"])
def test_alu_roofline_uses_derived_fp32_peak(bench, prec):
    r = bench.roofline(prec, 8.05, None, 5, _stats(), 40.0)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(0.1, rel=1e-3)


def test_committed_traffic_figure_is_read(bench):
    """profiles/traffic.txt holds the per-launch DRAM bytes of the bench's dominant kernel in the
    format the bench parses (kernel, workload, precision, bytes)."""
    entries = {}
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        parts = line.split()
        if len(parts) == 4:
            entries[tuple(parts[:3])] = float(parts[3])
    # the bench's default workload (C3) at its default arithmetic: traffic of the current kernel
    assert entries[("toeplitz", "C3", "bf16x3")] > 0
    traffic, pipe = bench.committed_counters("C3", "bf16x3")
    assert traffic == entries[("toeplitz", "C3", "bf16x3")]
    assert pipe is not None and 0 < pipe["value"] <= 100


def test_gate_is_per_problem(bench):
    """Each noisy solve is held to 1.5x its own oracle errors + 10 u32; noise-free solves to the
    absolute tolerances; a noisy solve without an oracle result does not count."""
    gate = bench.gate_from_oracle([(1e-5, 1e-3), (4e-5, 2e-3)])
    floor = 10 * 2.0 ** -24
    assert gate[0] == pytest.approx((1.5e-5 + floor, 1.5e-3 + floor))
    assert bench.passes_gate(True, gate, 0, 1.5e-5, 1.5e-3)
    assert not bench.passes_gate(True, gate, 0, 2.0e-5, 1e-3)      # within problem 1's threshold only
    assert bench.passes_gate(True, gate, 1, 2.0e-5, 1e-3)
    assert not bench.passes_gate(True, gate, 2, 0.0, 0.0)
    assert not bench.passes_gate(True, None, 0, 0.0, 0.0)
    assert bench.passes_gate(False, None, 0, 1e-6, 1e-5) and not bench.passes_gate(False, None, 0, 2e-6, 0.0)


def test_default_workload_is_the_precision_config(bench):
    assert bench.DEFAULT_BATCH["C3"] >= 1
    import sys
    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        assert bench.parse().config == "C3"
    finally:
        sys.argv = old


def test_single_problem_samples_cover_the_batched_workloads(bench):
    assert set(bench.SINGLE_SAMPLE) == {"C1", "C2", "C3", "C4"}
    assert all(v >= 1 for v in bench.SINGLE_SAMPLE.values())


def test_workload_recipes(bench):
    """C2 problems have the headline shape; C4 problems follow the batch recipe (n in 7..31,
    m in 2..12 and at most floor(n/2)^2), each with its own seed."""
    c2 = bench.make_problems("C2", 3)
    assert all((P.d, P.n, P.m) == (2, 63, 20) for P in c2)
    assert not np.array_equal(c2[0].grid, c2[1].grid)
    c4 = bench.make_problems("C4", 64)
    assert all(P.d == 2 and 7 <= P.n <= 31 and 2 <= P.m <= min(12, (P.n // 2) ** 2) for P in c4)
    assert len({P.n for P in c4}) > 1
