"""Host-side pieces of bench.py: the algorithmic work per launch and the roofline
arithmetic, including the accounting of skipped evaluations (a retry of a rejected
attempt keeps S(n^k): one forward-column and one row launch then return at once, and
one inverse pass only rescales k_1)."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32conv"])
def test_roofline_accounts_for_skipped_evaluations(bench, precision):
    sched = {"fft_lgn1": 8}
    ms, cnt = _prof(0)
    r0 = bench.roofline(precision, ms, cnt, 2, sched)
    assert r0["kernel"] == "rows"  # 60 x 40 us against 50 x 45 us
    fl, by = bench.algorithmic(1 << 17, 2, 8 if precision == "fp32conv" else 16, 8)
    work = fl["rows"] if precision == "fp64" else by["rows"]
    scale = 1e12 if precision == "fp64" else 1e9
    assert r0["achieved"] == pytest.approx(work / 40e-6 / scale)
    assert r0["frac"] == pytest.approx(r0["achieved"] / r0["peak"])
    ms, cnt = _prof(3)  # three of the 60 row launches did nothing
    r3 = bench.roofline(precision, ms, cnt, 2, sched)
    assert r3["achieved"] == pytest.approx(r0["achieved"] * (1 - 3 / 60))
    assert r3["profiled_evals_skipped"] == 3


def test_roofline_fused_pass_keeps_its_forward_work(bench):
    """A skipped evaluation removes only the inverse half of one fused launch."""
    ms = {"fwd_cols": 0.030, "rows": 0.030, "inv_cols": 0.0, "step": 0.0, "inv_fwd": 0.045, "inv_step": 0.039}
    cnt = {"fwd_cols": 10, "rows": 60, "inv_cols": 0, "step": 0, "inv_fwd": 50, "inv_step": 10, "skipped": 5}
    r = bench.roofline("fp64", ms, cnt, 2, {"fft_lgn1": 8})
    assert r["kernel"] == "inv_fwd"
    fl, _ = bench.algorithmic(1 << 17, 2, 16, 8)
    want = (50 * fl["inv_fwd"] - 5 * fl["inv_cols"]) / 50
    assert r["algorithmic_per_launch"] == pytest.approx(want)


def test_source_digest_ignores_comments(bench, tmp_path, monkeypatch):
    d = tmp_path / "paper_2407_16559_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "a.cu").write_text("int f() { return 1; }  // one\n/* block */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.src_digest()
    (d / "a.cu").write_text("int f() { return 1; }  // changed comment\n\n")
    assert bench.src_digest() == h1
    (d / "a.cu").write_text("int f() { return 2; }\n")
    assert bench.src_digest() != h1
