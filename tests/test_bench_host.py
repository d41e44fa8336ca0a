"""Host logic of bench.py (no GPU): the roofline arithmetic, the committed ncu
traffic figures and their source-hash guard, and the measured peaks file."""
import json

import pytest

import bench


def test_ntt_roofline_arithmetic():
    """achieved = butterflies per launch / mean launch time; the issue ceiling is the
    SM issue rate over the captured instructions a butterfly, the multiplier ceiling
    the sub-partition clock rate over the captured busy cycles a butterfly."""
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["ntt_fwd"]
    prof = {"launches": 10, "ms": 0.8, "ops": 10 * 4.0e7, "bytes": 10 * 8.0e7}
    r = bench.ntt_roofline(prof, {"sm_mhz": 2070.0}, {"butterfly_per_s": 1.0e12, "butterfly_k32_per_s": 2.0e12})
    assert r["bound"] == "alu" and r["unit"] == "Gbutterfly/s"
    assert r["achieved"] == pytest.approx(4.0e7 / 80e-6 / 1e9)
    assert r["peak"] == pytest.approx(1000.0)                  # the measured (general) butterfly rate
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.ntt_roofline(prof, None)["frac"] is None      # no measurement, no fraction
    if rec["source_sha256"] == bench.kernel_source_sha256("ntt_fwd"):
        issue = 152 * 4 * 32 * 2070e6 / rec["thread_instructions_per_butterfly"] / 1e9
        assert r["issue_peak"] == pytest.approx(issue)
        assert r["issue_frac"] == pytest.approx(r["achieved"] / issue)
        mul = 152 * 4 * 2070e6 / rec["fmaheavy_cycles_per_butterfly"] / 1e9
        assert r["multiplier_pipe_peak"] == pytest.approx(mul)
        assert r["multiplier_pipe_peak"] < r["issue_peak"]   # the multiplier binds first
    assert bench.ntt_roofline({"launches": 0, "ms": 0.0, "ops": 0, "bytes": 0}, None) is None


def test_committed_traffic_scales_and_guards(monkeypatch):
    """Traffic per launch is the captured DRAM/algorithmic ratio times the launch's
    algorithmic bytes, and None once the kernel's source no longer matches."""
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["ks_inner"]
    if rec["source_sha256"] == bench.kernel_source_sha256("ks_inner"):
        t = bench.committed_traffic("ks_inner", 1.0e8)
        assert t == pytest.approx(rec["dram_bytes"] / rec["algorithmic_bytes"] * 1.0e8)
        assert 0.9 < t / 1.0e8 < 1.1   # no re-reads in the captured launch
    monkeypatch.setattr(bench, "kernel_source_sha256", lambda k: "0" * 64)
    assert bench.committed_traffic("ks_inner", 1.0e8) is None
    assert bench.committed_traffic("no_such_kernel", 1.0e8) is None


def test_kernel_source_hash_covers_the_kernel_text():
    """The ks_inner hash is taken over the kernel's own source section only."""
    h1 = bench.kernel_source_sha256("ks_inner")
    h2 = bench.kernel_source_sha256("ks_inner")
    assert h1 == h2 and len(h1) == 64
    assert bench.kernel_source_sha256("ntt_fwd") != h1


def test_measured_peaks_are_positive():
    peak, kind = bench.measured_peaks()
    assert peak > 0 and isinstance(kind, str)


def test_key_switch_algorithmic_cost():
    """Explicit keys at 28 limbs (n = 2^16, alpha = 3, digits of 3): 8n [2 28 + 2 10 31 +
    2 28] bytes = 366 MiB; seeded keys stream one key part less; 18 and 9 limbs as the
    formula gives (162 and 54 MiB explicit)."""
    b, m = bench.ks_algorithmic(28, seeded=False)
    assert b == 8 * 65536 * (56 + 620 + 56)
    assert round(b / 2 ** 20) == 366
    bs, ms = bench.ks_algorithmic(28)
    assert b - bs == 8 * 65536 * 10 * 31 and ms == m
    assert round(bench.ks_algorithmic(18, seeded=False)[0] / 2 ** 20) == 162
    assert round(bench.ks_algorithmic(9, seeded=False)[0] / 2 ** 20) == 54
    assert m == 32768 * 16 * (310 + 56 + 6) + 65536 * (3 * 10 * 28 + 6 * 28 + 2 * 310)
