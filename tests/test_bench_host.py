"""Host-side arithmetic of bench.py, on the CPU: the form-weighted MUFU and
FMA-pipe ceilings the tensor-core loop's roofline is reported against, the
single-operation costs, the gradient loops' two counts, and the key that ties
the committed DRAM-traffic capture to the kernel source it was taken on."""
import json
import os
import shutil

import pytest

import bench

# the rates measured on a B300 (results, or pairs, per SM per clock)
RATES = {"sqrt": 16.0, "rsqrt": 16.0, "ex2": 32.0, "fma": 124.1, "rcp": 16.0,
         "pair_direct": 4.571, "pair_flat": 4.571, "pair_curved": 2.909}


def test_single_form_ceiling():
    """Every tensor-core form takes d on the FMA pipe: direct 2 sqrt + 1 exp2,
    flat 1 sqrt + 1 rcp + 1 exp2, curved 2 sqrt + 1 rcp + 1 exp2, from the
    single-operation rates."""
    expect = {"direct": 2 / 16.0 + 1 / 32.0, "flat": 1 / 16.0 + 1 / 16.0 + 1 / 32.0,
              "curved": 2 / 16.0 + 1 / 16.0 + 1 / 32.0}
    for form in ("direct", "flat", "curved"):
        best, mufu, fma = bench.tc_pair_ceiling(RATES, {form: 1000})
        assert mufu == pytest.approx(1.0 / expect[form])
        assert fma == pytest.approx(RATES["fma"] / bench.TC_FORM_COST[form][1])
        assert best == min(mufu, fma)
    # the direct form is bound by its special-function unit, not the FMA pipe
    best, mufu, fma = bench.tc_pair_ceiling(RATES, {"direct": 1})
    assert mufu < fma and best == mufu


def test_mixed_forms_share_the_clocks():
    """Pairs of each form cost 1 / rate SM-clocks, so the ceiling is the
    total of pairs over the total of clocks: between the forms' rates,
    unchanged when every count doubles, lower with more curved points."""
    counts = {"direct": 97904, "curved": 2096}
    _, mufu, _ = bench.tc_pair_ceiling(RATES, counts)
    curved = 1.0 / (3 / 16.0 + 1 / 32.0)
    assert curved < mufu < 6.4
    assert mufu == pytest.approx(100000 / (97904 / 6.4 + 2096 / curved))
    assert bench.tc_pair_ceiling(RATES, {k: 2 * v for k, v in counts.items()})[1] == pytest.approx(mufu)
    assert bench.tc_pair_ceiling(RATES, {"direct": 97904, "curved": 20960})[1] < mufu


def test_unmeasured_mix_falls_back_to_single_operations():
    single = {k: v for k, v in RATES.items() if not k.startswith("pair_")}
    assert bench.mix_cost(single, "direct") == pytest.approx(2 / 16.0 + 1 / 32.0)
    assert bench.mix_cost(single, "curved") == pytest.approx(2 / 16.0 + 1 / 16.0 + 1 / 32.0)
    # with the measured rates the mixes are additive: the single-operation sums
    # equal the mixes the probe times whole
    assert 1 / bench.single_op_cost(single, (3, 0, 1)) == pytest.approx(RATES["pair_direct"], rel=1e-3)
    assert 1 / bench.single_op_cost(single, (3, 2, 1)) == pytest.approx(RATES["pair_curved"], rel=1e-3)


def test_fp32_unit_loop_ceiling():
    """The FP32-unit loop keeps three MUFU square roots per pair; its 25 FP32
    operations leave the FMA pipe above the MUFU."""
    best, mufu, fma = bench.pair_ceiling(RATES, bench.FP32_PER_PAIR)
    assert mufu == pytest.approx(RATES["pair_direct"])
    single = {k: v for k, v in RATES.items() if not k.startswith("pair_")}
    assert bench.pair_ceiling(single, bench.FP32_PER_PAIR)[1] == pytest.approx(1 / (3 / 16.0 + 1 / 32.0))
    assert fma == pytest.approx(RATES["fma"] / 25)
    assert best == min(mufu, fma) == mufu


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    """A copy of the hashed kernel sources and the traffic capture."""
    src = os.path.join(bench.ROOT, "paper_2607_16946_b300", "csrc")
    dst = tmp_path / "paper_2607_16946_b300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("query_tc.cu", "tc_common.cuh", "query_common.cuh", "device_common.cuh", "internal.h"):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_kernel_hash_ignores_comments_not_code(tree):
    h0 = bench.kernel_source_sha()
    f = tree / "paper_2607_16946_b300" / "csrc" / "query_tc.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n", "\n\n", 3))
    assert bench.kernel_source_sha() == h0
    f.write_text(text + "\nstatic const int kExtra = 1;\n")
    assert bench.kernel_source_sha() != h0


def test_traffic_used_only_for_the_captured_source(tree):
    path = tree / "profiles" / "fwd_tc_dense_grid_traffic.json"
    assert bench.committed_traffic() is None                       # no capture
    path.write_text(json.dumps({"kernel_sha": bench.kernel_source_sha(), "dram_bytes_per_step": 1.0e9}))
    assert bench.committed_traffic() == 1.0e9
    path.write_text(json.dumps({"kernel_sha": "0" * 16, "dram_bytes_per_step": 1.0e9}))
    assert bench.committed_traffic() is None                       # taken on another source
    path.write_text("{not json")
    assert bench.committed_traffic() is None


def test_both_arms_describe_the_same_workload():
    c1, c4 = bench.workload_config(256 ** 3, 1), bench.workload_config(256 ** 3, 4)
    assert c1["Q"] == 256 ** 3 and c1["N"] == bench.N_POINTS and c1["workload"] == bench.WORKLOAD
    assert c1["parallelism"] == "single" and c4["parallelism"] == "replicas4"


def test_compact_summary_comes_from_the_legs():
    line = {"value": 1051.3, "e2e": {"value": 1046.5}, "roofline": {"frac": 0.8071},
            "mixed": {"sspd": {"value": 2500.0, "err_max_rel_diag": 1.2e-7,
                               "roofline": {"frac": 0.75}}, "note": "text"},
            "served": {"value": 700.0, "p50_ms": 500.0, "p99_ms": 2500.0},
            "cpu_baseline": {"value": 0.65}}
    s = bench.compact_summary(line)
    assert s["dense_grid"] == {"gpairs_s": 1051.0, "frac": 0.807, "e2e_gpairs_s": 1046.0}
    assert s["sspd"] == {"gpairs_s": 2500.0, "err_max": 1.2e-7, "frac": 0.75}
    assert s["served"]["p99_ms"] == 2500.0 and s["cpu_oracle_gpairs_s"] == 0.65
    assert "note" not in s


def test_gradient_rooflines_carry_both_counts():
    r = bench.grad_roofline(500.0, 37000.0, bench.GRAD_FP32_PER_PAIR, bench.GRAD_PLAN_FP32)
    assert r["frac"] == pytest.approx(500.0 / (37000.0 / 54))
    assert r["frac_plan_count"] == pytest.approx(500.0 / (37000.0 / 43))
    assert r["frac_plan_count"] < r["frac"]
    b = bench.grad_roofline(500.0, 37000.0, bench.BWD_FP32_PER_PAIR, bench.BWD_PLAN_FP32)
    assert b["frac_plan_count"] == pytest.approx(500.0 / (37000.0 / 46)) and "twice" in b["plan_count_basis"]


def test_radius_roofline_needs_a_capture_of_the_current_source(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2607_16946_b300", "csrc")
    dst = tmp_path / "paper_2607_16946_b300" / "csrc"
    dst.mkdir(parents=True)
    for f in set(bench.RADIUS_SOURCES):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.radius_issue_roofline(0.1, 148, 2032.0) is None
    path = tmp_path / "profiles" / "radius_large_cloud_counts.json"
    path.write_text(json.dumps({"kernel_sha": bench.kernel_source_sha(bench.RADIUS_SOURCES),
                                "warp_instructions_per_call": 6.0e10, "dram_bytes_per_call": 1.0e9}))
    r = bench.radius_issue_roofline(0.1, 148, 2032.0)
    assert r["achieved"] == pytest.approx(600.0) and r["peak"] == pytest.approx(4 * 148 * 2.032)
    assert r["frac"] == pytest.approx(600.0 / (4 * 148 * 2.032)) and r["traffic"] == 1.0e9
    path.write_text(json.dumps({"kernel_sha": "0" * 16, "warp_instructions_per_call": 6.0e10}))
    assert bench.radius_issue_roofline(0.1, 148, 2032.0) is None


def test_both_arms_print_the_same_config(monkeypatch, capsys):
    """The main arm and the reference (oracle) arm describe one workload with
    the same dict (the main arm puts how it runs it under its own key): the
    reference arm's printed line, with its timed oracle samples stubbed."""
    class Args:
        warmup, steps = 3, 2
    monkeypatch.setattr(bench, "_timed_oracle_sample", lambda *a, **k: (2048, 0.05))
    bench.run_reference(Args(), 0, 1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config(bench.GRID_RES ** 3, 1)
    c = line["config"]
    assert c["Q"] == bench.GRID_RES ** 3 and c["N"] == bench.N_POINTS
    assert "l2" in c and "engine" not in c and "precision" not in c
