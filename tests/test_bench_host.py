"""Host-side arithmetic of bench.py, on the CPU: the form-weighted MUFU
ceiling the tensor-core loop's roofline is reported against, its fallback to
single-operation costs, and the key that ties the committed DRAM-traffic
capture to the kernel source it was taken on."""
import json
import os
import shutil

import pytest

import bench

RATES = {"sqrt": 17.9, "rsqrt": 17.9, "ex2": 40.5, "fma": 128.5, "rcp": 17.8,
         "pair_direct": 4.71, "pair_flat": 4.71, "pair_curved": 2.96}


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
    assert mufu == pytest.approx(100000 / (97904 / 4.71 + 2096 / 2.96))
    assert bench.tc_pair_ceiling(RATES, {k: 2 * v for k, v in counts.items()})[1] == pytest.approx(mufu)
    assert bench.tc_pair_ceiling(RATES, {"direct": 97904, "curved": 20960})[1] < mufu


def test_unmeasured_mix_falls_back_to_single_operations():
    single = {k: v for k, v in RATES.items() if not k.startswith("pair_")}
    assert bench.mix_cost(single, "direct") == pytest.approx(3 / 17.9 + 1 / 40.5)
    assert bench.mix_cost(single, "curved") == pytest.approx(3 / 17.9 + 2 / 17.8 + 1 / 40.5)
    # the measured mix is slower than the sum of its parts on this part
    assert bench.mix_cost(RATES, "direct") > bench.mix_cost(single, "direct")


def test_fp32_unit_loop_ceiling():
    best, mufu, issue = bench.pair_ceiling(RATES, bench.INSTR_PER_PAIR)
    assert mufu == pytest.approx(4.71)
    assert issue == pytest.approx(128.5 / 29)
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
