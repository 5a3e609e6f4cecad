"""Host logic of bench.py (no GPU): the clock record keeps only the readings
taken inside the timed region and lists every throttle reason seen; a DRAM
traffic figure is reported only while its kernel's sources are unchanged."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_0905_2441_gb300 import build  # noqa: E402


def _line(sm, mx, power_cap="Not Active", thermal="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, Not Active, Not Active, {thermal}, {power_cap}"


def test_clock_summary_timed_region_and_reasons():
    c = bench.ClockSampler()
    c.lines = [_line(345, 2070), _line(2070, 2070, power_cap="Active"), _line(2070, 2070),
               _line(2055, 2070), "garbage"]
    c.start = 1  # the first reading came before the timed region
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines.append(_line(1500, 2070, thermal="Active"))
    assert "sw_thermal_slowdown" in c.summary()["reasons"]


def test_clock_summary_without_readings():
    c = bench.ClockSampler()
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []


def test_traffic_dropped_once_sources_change(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = ["is.cu", "device.cuh", "ctx.hpp"]
    entry = {"bytes_per_launch": 123, "sources": src, "source_digest": build.source_digest(src)}
    (prof / "traffic.json").write_text(json.dumps({"k_is_moments": entry,
                                                   "stale": dict(entry, source_digest="0")}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k_is_moments") == 123
    assert bench.profile_traffic("stale") is None
    assert bench.profile_traffic("absent") is None


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for name, e in d.items():
        assert e["bytes_per_launch"] > 0 and e["sources"], name
        build.source_digest(e["sources"])  # every listed source exists


def test_popmcmc_oracle_check_reports_zero_error_on_the_oracle_s_own_sweep():
    """The bench's error check against the oracle, fed a state whose stored
    log-likelihoods and one-sweep successor come from the oracle itself:
    no error, no differing chain (the check compares what it should)."""
    import oracle
    import synth
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    m = int(off[16])
    th = synth.population_particles(w.K, off, seed=4)[:, :m].copy()
    ll = oracle.gmm1d_loglik(w.data(), w.logw(), w.sigma, th)
    beta = synth.population_betas(off)[:m]
    rt, rl, _ = oracle.popmcmc_sweep(w.data(), w.logw(), w.sigma, (-10, 10), th, ll, beta,
                                     off[:17], w.scale, 3, 5)
    snap = {"theta": th, "ll": ll, "theta1": rt, "ll1": rl, "sweep": 5}
    r = bench.popmcmc_oracle_check(w, snap, n_chains=100, sample_pops=16)
    assert r["max_rel_loglik_err"] == 0.0
    assert r["sweep_replayed"]["chains_differing"] == 0
    assert r["sweep_replayed"]["populations_differing"] == 0
    # a planted change in one chain's successor is seen
    rt2 = rt.copy()
    rt2[0, 10] += 0.5
    r2 = bench.popmcmc_oracle_check(w, dict(snap, theta1=rt2), n_chains=100, sample_pops=16)
    assert r2["sweep_replayed"]["chains_differing"] == 1
