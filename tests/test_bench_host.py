"""Host-side arithmetic of bench.py, on the CPU: the form-weighted MUFU
ceiling the tensor-core loop's roofline is reported against, its fallback to
single-operation costs, and the key that ties the committed DRAM-traffic
capture to the kernel source it was taken on."""
import json
import os
import shutil

import pytest

import bench

# the rates measured on a B300 (results, or pairs, per SM per clock)
RATES = {"sqrt": 16.0, "rsqrt": 16.0, "ex2": 32.0, "fma": 124.1, "rcp": 16.0,
         "pair_direct": 4.571, "pair_flat": 4.571, "pair_curved": 2.909}


def test_single_form_ceiling_is_its_measured_mix():
    for form, key in bench.PAIR_MIX_KEYS.items():
        best, mufu, issue = bench.tc_pair_ceiling(RATES, {form: 1000})
        assert mufu == pytest.approx(RATES[key])
        assert issue == pytest.approx(RATES["fma"] / bench.TC_FORM_COST[form][1])
        assert best == min(mufu, issue)


def test_mixed_forms_share_the_clocks():
    """Pairs of each form cost 1 / rate SM-clocks, so the ceiling is the
    total of pairs over the total of clocks: between the forms' rates,
    unchanged when every count doubles, lower with more curved points."""
    counts = {"direct": 97904, "curved": 2096}
    _, mufu, _ = bench.tc_pair_ceiling(RATES, counts)
    assert RATES["pair_curved"] < mufu < RATES["pair_direct"]
    assert mufu == pytest.approx(100000 / (97904 / 4.571 + 2096 / 2.909))
    assert bench.tc_pair_ceiling(RATES, {k: 2 * v for k, v in counts.items()})[1] == pytest.approx(mufu)
    assert bench.tc_pair_ceiling(RATES, {"direct": 97904, "curved": 20960})[1] < mufu


def test_unmeasured_mix_falls_back_to_single_operations():
    single = {k: v for k, v in RATES.items() if not k.startswith("pair_")}
    assert bench.mix_cost(single, "direct") == pytest.approx(3 / 16.0 + 1 / 32.0)
    assert bench.mix_cost(single, "curved") == pytest.approx(3 / 16.0 + 2 / 16.0 + 1 / 32.0)
    # with the measured rates the mixes are additive: the single-operation sums
    # equal the measured mixes
    assert 1 / bench.mix_cost(single, "direct") == pytest.approx(RATES["pair_direct"], rel=1e-3)
    assert 1 / bench.mix_cost(single, "curved") == pytest.approx(RATES["pair_curved"], rel=1e-3)


def test_fp32_unit_loop_ceiling():
    best, mufu, issue = bench.pair_ceiling(RATES, bench.INSTR_PER_PAIR)
    assert mufu == pytest.approx(RATES["pair_direct"])
    assert issue == pytest.approx(RATES["fma"] / 29)
    assert best == min(mufu, issue)


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
