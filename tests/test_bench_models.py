"""Host logic of the benchmark's roofline reporting: the algorithmic work per
launch of each modelled kernel and the achieved rate derived from the live
launch timings (no GPU)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


INFO = dict(rank_sum_far=1000, near_rank_entries=50000, near_entries=8000, far_coupling=20 * 4096)


def test_factored_models_count_complex_macs(bench):
    m = bench.kernel_models(dict(INFO, near_expanded=0, far_expanded=0), Ls=129, p=64, tensor_cores=0)
    assert m["far_coupling"]["work"] == 8.0 * 1000 * 64 * 64 * 129
    assert m["near_apply"]["work"] == 8.0 * 50000 * 129
    # float-float: 48 FP32 instructions per complex multiply-add, 2 flops each
    assert m["far_exact"]["work"] == 2.0 * 48 * 1000 * 64 * 64 * 129
    assert all(v["bound"] == "alu" and v["unit"] == "TFLOP/s" for v in m.values())


def test_tensor_and_expanded_models(bench):
    m = bench.kernel_models(dict(INFO, near_expanded=1, far_expanded=1), Ls=129, p=64, tensor_cores=2)
    assert m["far_coupling"]["bound"] == "tensor"
    peak, _ = bench.tf32_peak()
    assert m["far_coupling"]["peak"] == pytest.approx(peak)
    m1 = bench.kernel_models(dict(INFO, near_expanded=1, far_expanded=1), Ls=129, p=64, tensor_cores=1)
    pk, _ = bench._peaks()
    assert m1["far_coupling"]["peak"] == pytest.approx(pk.get("bf16_tflops_sustained", pk["bf16_tflops"]))
    assert m1["far_coupling"]["work"] == 8.0 * 1000 * 64 * 64 * 129
    assert m["near_apply"]["bound"] == "hbm" and m["near_apply"]["work"] == 8.0 * 8000 * 129
    assert m["near_exact"]["work"] == 16.0 * 8000 * 129
    assert m["far_exact"]["bound"] == "hbm" and m["far_exact"]["work"] == 16.0 * 20 * 4096 * 129


def test_roofline_entry_rates(bench):
    mdl = dict(bound="hbm", peak=8000.0, unit="GB/s", work=4.0e9, what="", peak_source="")
    r = bench.roofline_entry("k", 4, 8.0, mdl)  # 4 launches, 8 ms in total: 2 ms each
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(4.0e9 / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 8000.0)
    mdl = dict(bound="alu", peak=80.0, unit="TFLOP/s", work=1.0e12, what="", peak_source="")
    r = bench.roofline_entry("k", 10, 100.0, mdl)
    assert r["achieved"] == pytest.approx(1.0e12 / 1e-2 / 1e12)


def test_time_weighted_fraction(bench):
    models = {"a": dict(bound="hbm", peak=100.0, unit="GB/s", work=1.0e9, what="", peak_source=""),
              "b": dict(bound="alu", peak=10.0, unit="TFLOP/s", work=1.0e12, what="", peak_source="")}
    prof = {"a": (10, 100.0), "b": (1, 300.0), "c": (5, 1.0)}
    fa = bench.roofline_entry("a", 10, 100.0, models["a"])["frac"]
    fb = bench.roofline_entry("b", 1, 300.0, models["b"])["frac"]
    tw = bench.time_weighted_frac(prof, models)
    assert tw["frac"] == pytest.approx((100.0 * fa + 300.0 * fb) / 400.0)
    assert tw["ms"] == pytest.approx(400.0) and tw["kernels"] == ["a", "b"]


def test_maca_and_arnoldi_models(bench):
    info = dict(INFO, near_expanded=1, far_expanded=1, nt=5120, maca_slice_evals=4.0e9,
                maca_fibre_evals=1.0e9)
    sinfo = dict(iterations=100, arnoldi_vectors=20000, arnoldi_freq_steps=1200)
    lps = {"maca_slice": 16.0, "maca_fibre": 16.0}
    m = bench.kernel_models(info, Ls=129, p=64, tensor_cores=1, sinfo=sinfo, launches_per_step=lps)
    k = bench.MACA_FF_INSTR_PER_EVAL
    assert m["maca_slice"]["bound"] == "alu" and m["maca_slice"]["work"] == 4.0e9 * k / 16.0
    assert m["maca_fibre"]["work"] == 1.0e9 * k / 16.0
    assert m["maca_slice"]["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    # basis read four times and w eight times per active frequency and step
    assert m["arnoldi"]["bound"] == "hbm"
    assert m["arnoldi"]["work"] == (4.0 * 20000 + 8.0 * 1200) * 5120 * 16.0 / 100
    # the streams count the frequencies they read: active ones per Arnoldi
    # step, unconverged ones per restart
    assert m["near_apply"]["work"] == pytest.approx(8.0 * INFO["near_entries"] * 1200 / 100)
    sinfo2 = dict(sinfo, restarts=4, restart_freq_applies=300)
    m2 = bench.kernel_models(info, Ls=129, p=64, tensor_cores=1, sinfo=sinfo2, launches_per_step=lps)
    assert m2["near_exact"]["work"] == pytest.approx(16.0 * INFO["near_entries"] * 75.0)
    assert m2["far_exact"]["work"] == pytest.approx(16.0 * INFO["far_coupling"] * 75.0)
    # without counts the models are left out, and the streams count every frequency
    m0 = bench.kernel_models(info, Ls=129, p=64, tensor_cores=1)
    assert "maca_slice" not in m0 and "arnoldi" not in m0
    assert m0["near_apply"]["work"] == 8.0 * INFO["near_entries"] * 129


def test_mot_models(bench):
    info = dict(nt=1280, n_leaves=64, rank_sum_far=100, rank_sum_near=50, near_rank_entries=40000)
    N = 64
    m = bench.mot_models(info, N, {"mot_history": 64.0, "mot_step": 65.0})
    lags = N * (N + 1) / 2
    per_lag = 100 * 64 + 50 * 20.0
    per_step = 100 * 4096 + 40000
    k = bench.MOT_FF_INSTR_PER_MAC
    assert m["mot_history"]["work"] == pytest.approx(k * (per_lag * lags + per_step * N) / 64.0)
    assert m["mot_history"]["bound"] == "alu" and m["mot_history"]["unit"] == "Tinst/s"
    assert m["mot_step"]["work"] == pytest.approx(8.0 * 1280 * 1280 * 65 / 65.0)
    assert abs(bench.cqm_R(N) ** (N + 1) - 1e-5) < 1e-12


def test_tc2_traffic_scales_image_bytes(bench, monkeypatch):
    # no capture of the current kernel: no traffic figure
    monkeypatch.setattr(bench, "TC2_CAPTURE", None)
    assert bench.tc2_traffic(dict(rank_sum_far=100, tc_single_terms=10)) is None
    # images counted exactly (32 KB per three-product term, 16 KB per single
    # one); the capture's other bytes scaled per rank term
    cap = dict(dram=1000 * 32768.0 + 200 * 16384.0 + 1200 * 100.0, terms=1200, single=200)
    monkeypatch.setattr(bench, "TC2_CAPTURE", cap)
    t = bench.tc2_traffic(dict(rank_sum_far=3000, tc_single_terms=1000))
    assert t == pytest.approx(2000 * 32768.0 + 1000 * 16384.0 + 3000 * 100.0)
