"""Host-side pieces of bench.py: the algorithmic work per launch, the compulsory bytes
per attempt, the roofline arithmetic (including the accounting of skipped evaluations:
a retry of a rejected attempt keeps S(n^k), so one forward-column and one row launch
then return at once and one inverse pass only rescales k_1) and the error bound used
against the oracle's stored trajectories."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_counts(bench):
    M, T = 1 << 17, 2
    fl, by = bench.algorithmic(M, T, 16, 8)
    Mp = 1 << 17
    assert fl["fwd_cols"] == T * 5.0 * Mp * 8
    assert fl["rows"] == (T + 1) * 5.0 * Mp * (9 + 1)
    assert fl["inv_fwd"] == fl["inv_cols"] + fl["fwd_cols"]
    # the whole evaluation: (T + 1) transforms of log2 Mp levels plus the split / merge
    assert fl["fwd_cols"] + fl["rows"] + fl["inv_cols"] == (T + 1) * 5.0 * Mp * (17 + 1)
    assert by["rows"] == (T + 1) * 16 * Mp


def _prof(skipped):
    ms = {"fwd_cols": 0.030, "rows": 0.040, "inv_cols": 0.0, "step": 0.0, "inv_fwd": 0.045, "inv_step": 0.039}
    cnt = {"fwd_cols": 10, "rows": 60, "inv_cols": 0, "step": 0, "inv_fwd": 50, "inv_step": 10, "skipped": skipped}
    return ms, cnt


def test_roofline_fp64_against_measured_fp64_rate(bench):
    sched = {"fft_lgn1": 8}
    ms, cnt = _prof(0)
    peaks = {"fp64_tflops": 1.2}
    r0 = bench.roofline("fp64", ms, cnt, 2, sched, peaks)
    assert r0["kernel"] == "rows"  # 60 x 40 us against 50 x 45 us
    fl, _ = bench.algorithmic(1 << 17, 2, 16, 8)
    assert r0["achieved"] == pytest.approx(fl["rows"] / 40e-6 / 1e12)
    assert r0["peak"] == 1.2 and r0["frac"] == pytest.approx(r0["achieved"] / 1.2)
    assert "measured" in r0["peak_source"]
    ms, cnt = _prof(3)  # three of the 60 row launches did nothing
    r3 = bench.roofline("fp64", ms, cnt, 2, sched, peaks)
    assert r3["achieved"] == pytest.approx(r0["achieved"] * (1 - 3 / 60))
    assert r3["profiled_evals_skipped"] == 3
    rd = bench.roofline("fp64", ms, cnt, 2, sched, {})  # no live figure: derived, and labelled so
    assert rd["peak"] == pytest.approx(bench.FP64_DERIVED_TFLOPS) and "derived" in rd["peak_source"]


def test_roofline_fused_pass_keeps_its_forward_work(bench):
    """A skipped evaluation removes only the inverse half of one fused launch."""
    ms = {"fwd_cols": 0.030, "rows": 0.030, "inv_cols": 0.0, "step": 0.0, "inv_fwd": 0.045, "inv_step": 0.039}
    cnt = {"fwd_cols": 10, "rows": 60, "inv_cols": 0, "step": 0, "inv_fwd": 50, "inv_step": 10, "skipped": 5}
    r = bench.roofline("fp64", ms, cnt, 2, {"fft_lgn1": 8}, {"fp64_tflops": 1.2})
    assert r["kernel"] == "inv_fwd"
    fl, _ = bench.algorithmic(1 << 17, 2, 16, 8)
    want = (50 * fl["inv_fwd"] - 5 * fl["inv_cols"]) / 50
    assert r["algorithmic_per_launch"] == pytest.approx(want)


def test_compulsory_bytes_per_attempt(bench):
    """RKF45, T distinct weight vectors: every stage reads the state, the earlier stage
    vectors and the weights once and writes k_i; the final combination reads the state
    and 5 stage vectors and writes the new state (and, reduced forms, its shadow)."""
    for prec, w, sh in (("fp64", 8, 0), ("df64", 8, 8)):
        a, per = bench.compulsory(prec, 2)
        assert a == 6 * w + 15 * w + 6 * 2 * w + 6 * w + 8 + 5 * w + 8 + sh
        assert per["rows"] == 0.0
    a, _ = bench.compulsory("fp64", 4)  # no shared transforms: T = 2R = 4 at R = 2
    assert a == 464  # 464 M bytes per attempt with FP64 weights
    a, _ = bench.compulsory("fp32conv", 2)
    assert a == 6 * 4 + 15 * 4 + 6 * 2 * 4 + 6 * 4 + 8 + 5 * 4 + 8 + 4
    # the kernel shares of one attempt add up to the attempt
    a, per = bench.compulsory("fp64", 2)
    assert per["fwd_cols"] + 5 * per["inv_fwd"] + per["inv_step"] == pytest.approx(a)


def test_roofline_reduced_forms_use_compulsory_bytes(bench):
    ms = {"fwd_cols": 0.030, "rows": 0.010, "inv_cols": 0.0, "step": 0.0, "inv_fwd": 0.020, "inv_step": 0.039}
    cnt = {"fwd_cols": 10, "rows": 60, "inv_cols": 0, "step": 0, "inv_fwd": 50, "inv_step": 10, "skipped": 0}
    r = bench.roofline("fp32conv", ms, cnt, 2, {"fft_lgn1": 9}, {})
    assert r["kernel"] == "inv_fwd" and r["bound"] == "hbm"
    _, per = bench.compulsory("fp32conv", 2)
    assert r["algorithmic_per_launch"] == pytest.approx(per["inv_fwd"] * (1 << 17))
    assert r["achieved"] == pytest.approx(per["inv_fwd"] * (1 << 17) / 20e-6 / 1e9)
    assert r["fft_pass_bytes_per_launch"] > r["algorithmic_per_launch"]


def test_attempt_hbm_fraction(bench):
    h = bench.attempt_hbm("fp64", 2, 1 << 17, 0.5)
    a, _ = bench.compulsory("fp64", 2)
    assert h["compulsory_bytes"] == a * (1 << 17)
    assert h["gbs"] == pytest.approx(a * (1 << 17) / 0.5e-3 / 1e9)
    assert h["frac"] == pytest.approx(h["gbs"] / h["peak_gbs"])


def test_relative_error_bound_is_an_upper_bound(bench):
    import numpy as np
    rng = np.random.default_rng(3)
    ref = rng.uniform(0, 1, 300)
    got = ref + rng.normal(0, 1e-6, 300)
    exact = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    b = bench.rel_err_bound(got[:100], float(np.linalg.norm(got[100:])), ref[:100], float(np.linalg.norm(ref[100:])))
    assert b >= exact
    full = bench.rel_err_bound(got, 0.0, ref, 0.0)
    assert full == pytest.approx(exact)


def test_source_digest_ignores_comments(bench, tmp_path, monkeypatch):
    """The digest follows the kernel headers' code, not their comments, and not the host
    sources."""
    d = tmp_path / "paper_2407_16559_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "a.cuh").write_text("int f() { return 1; }  // one\n/* block */\n")
    (d / "host.cu").write_text("int g() { return 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.src_digest()
    (d / "a.cuh").write_text("int f() { return 1; }  // changed comment\n\n")
    assert bench.src_digest() == h1
    (d / "host.cu").write_text("int g() { return 2; }\n")
    assert bench.src_digest() == h1
    (d / "a.cuh").write_text("int f() { return 2; }\n")
    assert bench.src_digest() != h1
