"""Host-side logic of bench.py, without a GPU: the per-step percentiles, the
comment-insensitive hash that guards the committed ncu counters, the
issue-bound roofline arithmetic, and the clock sampler's filtering of the
samples to the timed region."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_percentiles_nearest_rank(bench):
    p = bench.percentiles([5.0, 1.0, 3.0, 2.0, 4.0, 6.0, 7.0, 8.0, 9.0, 10.0])
    assert p["n"] == 10 and p["p10"] == 2.0 and p["p90"] == 9.0
    assert p["p50"] in (5.0, 6.0)
    assert bench.percentiles([]) is None
    one = bench.percentiles([3.5])
    assert one["p10"] == one["p50"] == one["p90"] == 3.5


def test_code_only_ignores_comments_and_spacing(bench):
    a = 'int f(int x) {\n  // a comment\n  return x + 1; /* block */\n}\n'
    b = 'int f(int x)   {\n\n    return x + 1;   }'  # the same tokens, other spacing
    c = 'int f(int x) { return x + 2; }'
    s = 'const char *s = "// not a comment";'
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
    assert "// not a comment" in bench._code_only(s)


def test_sources_hash_matches_committed_counters(bench):
    """The committed trace counters were taken on the current trace sources
    (else the bench line would report no achieved issue rate)."""
    h = bench.sources_hash(bench.TRACE_SOURCES)
    e = bench.ncu_counters("trace_kernel", "room256_1080p_f32")
    assert e, "profiles/roofline_traffic.json does not match the trace sources (hash %s)" % h
    assert e["sources"] == h


def test_issue_roofline_arithmetic(bench, monkeypatch):
    counters = {"warp_inst_per_launch": 5.0e9, "warp_inst_per_sample": 9.5,
                "dram_bytes_per_launch": 1.0e8, "l1tex_bytes_per_launch": 2.0e10,
                "l1tex_throughput_pct": 50.0}
    monkeypatch.setattr(bench, "ncu_counters", lambda k, w: counters)
    clocks = {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0}
    r = bench.issue_roofline("trace_kernel", "w", 5.0, clocks, 150, 1.0e11, 7000.0, "measured")
    peak = 150 * bench.ISSUE_PER_SM_PER_CLOCK * 2000.0e6 / 1e9
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(5.0e9 / 5.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] == 1.0e8
    assert r["dram"]["achieved_gbs"] == pytest.approx(1.0e8 / 5.0e-3 / 1e9)
    assert r["gather_delivery"]["of_hbm_peak"] == pytest.approx(1.0e11 / 5.0e-3 / 1e9 / 7000.0)
    # without counters taken on the current sources: no achieved figure
    monkeypatch.setattr(bench, "ncu_counters", lambda k, w: {})
    r = bench.issue_roofline("trace_kernel", "w", 5.0, clocks, 150, 1.0e11, 7000.0, "measured")
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None


def test_clock_sampler_keeps_samples_of_the_timed_region(bench):
    cs = bench.ClockSampler(0)
    cs.proc = None  # no nvidia-smi here: feed lines directly
    row = "0, {mhz}, 2070, 900, 0x0, Not Active, Not Active, Not Active, {cap}"
    cs.lines = [(1.0, row.format(mhz=345, cap="Not Active")),      # idle, before
                (2.0, row.format(mhz=2070, cap="Not Active")),
                (2.1, row.format(mhz=2040, cap="Active")),
                (9.0, row.format(mhz=600, cap="Not Active"))]      # after
    class _P:
        def terminate(self): pass
        def wait(self, timeout=None): pass
    class _T:
        def join(self, timeout=None): pass
    cs.proc, cs.t = _P(), _T()
    r = cs.stop(1.5, 3.0)
    assert r["samples"] == 2 and r["sm_mhz"] == pytest.approx(2055.0)
    assert r["reasons"] == ["sw_power_cap"] and r["sm_max_mhz"] == 2070.0
    r = cs.stop(5.0, 6.0)  # nothing inside: every sample counts
    assert r["samples"] == 4
