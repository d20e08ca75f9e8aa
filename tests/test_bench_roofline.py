"""The roofline arithmetic of bench.py, recomputed by hand from its
definition: 6n flops per MP step against 152 SMs x 128 FP32 lanes x 2 flops
x 2070 MHz; 4n^2 flops per correlated leaf against the BF16 peak; the
latency view from the longest pursuit; the traffic ratio."""
import pytest

import bench

PEAKS = {"bf16_tflops": 1917.6, "hbm_gbs": 6798.6}


def _stats(level, attempts=0, iters=0, longest=0):
    z = [0] * 8
    st = {"attempts_per_level": list(z), "iterations_per_level": list(z), "max_leaf_steps_per_level": list(z)}
    st["attempts_per_level"][level] = attempts
    st["iterations_per_level"][level] = iters
    st["max_leaf_steps_per_level"][level] = longest
    return st


def test_pursuit_roofline_counts_6n_flops_per_step_against_the_fp32_fma_peak():
    # 20 launches of the side-64 pursuit, 134 126 steps each, 1.0153 ms each
    st = _stats(0, attempts=256 * 20, iters=134126 * 20, longest=1024)
    r = bench.roofline("mp_b64", 20, 20 * 1.0153, st, PEAKS, "measured", 2070.0, 64, step_floor_ns=966.5)
    n = 64 * 64
    achieved = 6 * n * 134126 / 1.0153e-3 / 1e12
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(80.54784)
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / peak)
    assert r["frac"] == pytest.approx(0.0403, abs=5e-4)
    lat = r["latency"]
    assert lat["ns_per_step_of_longest"] == pytest.approx(1.0153e6 / 1024)
    assert lat["chain_frac"] == pytest.approx(1024 * 966.5 / 1.0153e6)


def test_correlation_roofline_counts_4n2_flops_per_leaf_against_bf16():
    st = _stats(0, attempts=50910 * 3)
    r = bench.roofline("corr_septc_b64", 3, 3 * 10.29, st, PEAKS, "measured", 2070.0, 64)
    n = 64 * 64
    achieved = 4 * n * n * 50910 / 10.29e-3 / 1e12
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / 1917.6)
    assert r["separable_flops_per_leaf"] == 8 * 64 ** 3
    assert r["frac_separable_count"] == pytest.approx(8 * 64 ** 3 * 50910 / 10.29e-3 / 1e12 / 1917.6)


def test_one_family_correlation_counts_half_the_work():
    # the DCT-II family alone (the tensor-core half of the side-64 split)
    st = _stats(0, attempts=50910)
    r = bench.roofline("corr_septc_dct_b64", 1, 5.0, st, PEAKS, "measured", 2070.0, 64)
    n = 64 * 64
    assert r["achieved"] == pytest.approx(2 * n * n * 50910 / 5.0e-3 / 1e12)
    assert r["separable_flops_per_leaf"] == 4 * 64 ** 3
    kpad = n
    assert r["algorithmic_bytes"] == pytest.approx(2.0 * n * n + 50910 * (2.0 * kpad + 8.0 * n))
    both = bench.roofline("corr_septc_b64", 1, 5.0, st, PEAKS, "measured", 2070.0, 64)
    assert both["achieved"] == pytest.approx(2 * r["achieved"])
    assert both["tensor_flops_issued_per_leaf"] == 2 * r["tensor_flops_issued_per_leaf"]


def test_fp32_form_issues_one_fma_per_updated_correlation():
    st = _stats(1, attempts=10, iters=1000, longest=200)
    exact = bench.roofline("mp_b32", 1, 0.1, st, PEAKS, "measured", None, 64)
    fp32 = bench.roofline("mp_fp32_b32", 1, 0.1, st, PEAKS, "measured", None, 64)
    assert exact["issued_fp32_ops_per_alg_flop"] == pytest.approx(2.5)
    assert fp32["issued_fp32_ops_per_alg_flop"] == pytest.approx(1.0 / 6.0)
    assert exact["achieved"] == pytest.approx(6 * 32 * 32 * 1000 / 1e-4 / 1e12)


def test_gather_roofline_counts_bytes_against_hbm():
    st = _stats(2, attempts=4096)
    r = bench.roofline("gather_b16", 1, 0.01, st, PEAKS, "measured", None, 64)
    byts = 4096 * (256 + 2 * 256 + 4)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(byts / 1e-5 / 1e9)


def test_critical_path_sums_the_longest_pursuits():
    st = {"max_leaf_steps_per_level": [1024, 256, 64, 16, 4, 0, 0, 0]}
    assert bench.critical_path(st) == 1364


def test_profiled_traffic_matches_workload_and_scales_by_leaves(tmp_path, monkeypatch):
    import hashlib
    import json
    src = tmp_path / "paper_2605_09190_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_bytes(b"kernel source")
    (tmp_path / "profiles").mkdir()
    entry = {"dram_bytes_per_launch": 1000, "sources": ["k.cu"],
             "sources_sha256": hashlib.sha256(b"kernel source").hexdigest(),
             "workload": "uneven64", "leaves_per_launch": 100}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k_b64": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k_b64", "uneven64", 100) == 1000
    assert bench.profiled_traffic("k_b64", "uneven64", 25) == 250
    assert bench.profiled_traffic("k_b64", "sweep512", 100) is None     # captured on another workload
    assert bench.profiled_traffic("other_b64", "uneven64", 100) is None
    (src / "k.cu").write_bytes(b"kernel source, changed")
    assert bench.profiled_traffic("k_b64", "uneven64", 100) is None     # sources changed since the capture
