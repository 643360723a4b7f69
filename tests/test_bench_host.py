"""Host logic of bench.py that needs no GPU: the clock record built from
nvidia-smi rows (median SM clock, maximum, throttle reasons seen, malformed
rows skipped), the per-workload default step counts, and the protocol of the
warm-start training runs (driven through a recording stand-in for the
context)."""
import sys

import bench


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, pcap]


def test_clock_summary():
    s = bench.ClockSampler(0)
    s.rows = [_row(2070, 2070), _row(2040, 2070, pcap="Active"), _row(2070, 2070), ["garbage"],
              _row("[N/A]", 2070)]
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_throttling():
    s = bench.ClockSampler(0)
    s.rows = [_row(1500, 2070, hwt="Active"), _row(1400, 2070, swt="Active"), _row(1600, 2070, hw="Active")]
    out = s.summary()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0)
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_default_steps(monkeypatch):
    for argv, steps in ([[], 5], [["--workload", "pt27"], 50], [["--workload", "batch16"], 5],
                        [["--impl", "reference"], 3], [["--steps", "7"], 7]):
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        assert bench.parse().steps == steps


def test_default_steps_warm64(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "warm64"])
    assert bench.parse().steps == 3


class _FakeCtx:
    """Records the calls the warm-start training runs make (no GPU)."""

    def __init__(self):
        self.calls, self.logging, self.alns = [], False, []

    def mlp_enable(self, on):
        self.calls.append(("mlp", on))

    def load_alignment(self, codes):
        self.alns.append(codes.shape)
        return len(self.alns) - 1

    def set_model(self, aid, exch, freqs, alpha, ncat):
        self.calls.append(("model", aid, ncat))

    def hill_climb(self, aid, edges, lengths):
        self.calls.append(("climb", aid, len(edges), self.logging))
        return {"edges": edges, "lengths": lengths}

    def training_log(self, on, capacity=0):
        self.logging = on

    def begin(self, aid, edges, lengths, thr):
        self.calls.append(("begin", aid, len(edges), thr, self.logging))
        return 0.0, {"edges": edges[:1], "lengths": lengths[:1]}

    def expand(self, aid, edges, lengths, thr, lmax):
        self.calls.append(("expand", aid, len(edges), thr, self.logging))
        return lmax, {"edges": edges[:0], "lengths": lengths[:0]}  # the search ends


def test_training_runs_protocol():
    """Every 5th logged run is a 7-taxon x 500-site JC69 search (one category,
    infinite threshold, one random start); the others are 27-taxon x 2000-site
    GTR+G4 searches (4 categories, threshold 10) from 8 hill-climbs, which are
    not logged; the network stays off; every round is logged."""
    ctx = _FakeCtx()
    runs = bench.log_training_runs(ctx, 0, 5)
    assert runs == {"jc7_exhaustive": 1, "gtr27_climbed": 4}
    assert ctx.calls[0] == ("mlp", False)
    assert [s[0] for s in ctx.alns] == [27, 27, 27, 27, 7]
    climbs = [c for c in ctx.calls if c[0] == "climb"]
    assert [c[1] for c in climbs] == [0, 1, 2, 3] and all(c[2] == 8 and not c[3] for c in climbs)
    models = {c[1]: c[2] for c in ctx.calls if c[0] == "model"}
    assert models == {0: 4, 1: 4, 2: 4, 3: 4, 4: 1}
    searches = [c for c in ctx.calls if c[0] in ("begin", "expand")]
    assert all(c[4] for c in searches)  # logged
    assert {c[3] for c in searches if c[1] < 4} == {bench.TRAIN_THRESH}
    assert {c[3] for c in searches if c[1] == 4} == {float("inf")}
    assert not ctx.logging
