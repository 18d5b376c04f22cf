"""Host-side helpers of bench.py (no GPU): the achieved-rate report of the two-population
leg and the traffic-record lookup, so that an edit cannot break the JSON line."""
import importlib.util
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_two_pop_rates_from_a_traced_step(bench):
    share = {"basis_ionize": {"ms": 42.1}, "forward_fft": {"ms": 6.6}, "ps_plane": {"ms": 20.0},
             "tables": {"ms": 8.8}}
    r = bench.two_pop_rates(share, 24, 4797, 256, 500.0, 192)
    assert set(r) == {"contraction", "pencil_r2c", "ps_line_passes"}
    # useful flops: 2 x rank per cell and radius task
    assert r["contraction"]["achieved"] == pytest.approx(2 * 24 * 256 ** 3 * 4797 / 42.1e-3 / 1e12)
    # power spectrum: 3 passes over the planes below k_hi = 1.5 / Mpc (k_f = 2 pi / 500)
    planes = math.ceil(1.5 / (2 * math.pi / 500.0))
    assert r["ps_line_passes"]["achieved"] == pytest.approx(192 * 3 * planes * 256 * 256 * 8 / 20.0e-3 / 1e9)
    for v in r.values():
        assert 0 < v["frac"] < 2 and v["peak"] > 0


def test_two_pop_rates_without_classes(bench):
    assert bench.two_pop_rates({}, 24, 0, 256, 500.0, 0) == {}


def test_traffic_record_used_only_for_its_sources(bench):
    # the committed ncu record feeds roofline.traffic (bytes per unit x the launch's units) only
    # while the class's sources hash to the recorded value and the grid is the recorded one
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        rec = json.load(f)
    for cls, e in rec["per_class"].items():
        assert e["bytes_per_unit"] == pytest.approx((e["read"] + e["write"]) / e["units"])
        got = bench.ncu_launch_traffic(cls, 10.0, e.get("ps_split"))
        if e["source_hash"] == bench.class_source_hash(cls) and e["n"] == bench.N:
            assert got == pytest.approx(10.0 * e["bytes_per_unit"])
        else:
            assert got is None
    assert bench.ncu_launch_traffic("no_such_class", 1.0) is None
    assert bench.ncu_launch_traffic("ps_plane", 1.0, 2) is None   # another tiling's kernels


def test_f16_column_chunks_follows_the_placement_rule(bench):
    # the executed-FLOP figure counts 256-column chunks of the flag contraction: walkers'
    # radii above R_cell in groups of 32 (one group at least), a two-group walker starting on
    # an even group; checked here against the columns laid out one by one
    def layout(ladders):
        cols = []
        for w, nr in enumerate(ladders):
            width = max(nr - 1, 0)
            ng = max(1, -(-width // 32))
            if ng == 2 and (len(cols) // 32) % 2:
                cols += [None] * 32
            cols += [w] * width + [None] * (ng * 32 - width)
        return -(-len(cols) // 256)
    assert bench.f16_column_chunks([]) == 0 == layout([])
    for ladders in ([1], [2] * 8, [33] * 8, [17, 31, 40, 2, 64, 33, 1], [40, 9] * 11, list(range(1, 65))):
        assert bench.f16_column_chunks(ladders) == layout(ladders), ladders


def test_reference_arm_prints_the_contract_line():
    # `bench.py --impl reference` times the FP64 oracle on the host cores (one realization here)
    # and prints one JSON line with the fields the driver reads; it needs no GPU
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["n"] == 128 and d["config"]["z"] == [8.0, 9.0, 10.0]
