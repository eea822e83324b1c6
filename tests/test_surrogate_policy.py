"""Host logic of the surrogate rollout policy (audit every A windows, restore
and re-run by the LB on a failed audit, back-off), against a fake solver that
records what it is asked to do."""
from __future__ import annotations

from paper_2209_01444_gb300 import surrogate as S


class FakeSim:
    """Tracks the step count and which windows the state came from."""

    def __init__(self, verdicts):
        self.steps = 0
        self.source = []      # per window: "nn" or "lb"
        self.snap = None
        self.verdicts = list(verdicts)  # accepted flags of successive audits
        self.log = []

    def snapshot_save(self, slot=0):
        self.snap = (self.steps, list(self.source))
        self.log.append(("save", self.steps))

    def snapshot_restore(self, slot=0):
        self.steps, self.source = self.snap[0], list(self.snap[1])
        self.log.append(("restore", self.steps))

    def step(self, n):
        assert n % 50 == 0
        self.steps += n
        self.source += ["lb"] * (n // 50)
        self.log.append(("lb", n))

    def surrogate_advance(self, net, K, tol, audit, cx, cy, orient=0.0):
        self.steps += K
        if not audit:
            self.source.append("nn")
            return {"audited": False, "accepted": False, "tip_err": 0.0}
        self.source.append("lb")  # an audited window keeps the LB result
        ok = self.verdicts.pop(0)
        return {"audited": True, "accepted": ok, "tip_err": self.err if ok else 3.0}

    err = 0.01


def test_all_audits_pass():
    sim = FakeSim([True] * 10)
    st = S.rollout(sim, None, windows=12, K=50, tip_tol=1.0, audit_every=4, backoff=2, cx=0, cy=0)
    assert sim.steps == 600
    assert sim.source == (["nn"] * 3 + ["lb"]) * 3
    assert st["surrogate"] == 9 and st["audited"] == 3 and st["rejected"] == 0


def test_failed_audit_reruns_the_stretch_and_backs_off():
    sim = FakeSim([True, False, True, True])
    st = S.rollout(sim, None, windows=14, K=50, tip_tol=1.0, audit_every=3, backoff=2, cx=0, cy=0)
    assert sim.steps == 700
    # windows 0-2 pass; 3-5 fail the audit and are re-run by the LB; 6-7 back off;
    # 8-10 pass; 11-13: the last window is always audited
    assert sim.source == ["nn", "nn", "lb"] + ["lb"] * 3 + ["lb"] * 2 + ["nn", "nn", "lb"] + ["nn", "nn", "lb"]
    assert st["rejected"] == 1 and st["lb_rerun"] == 2 and st["lb_backoff"] == 2
    assert st["surrogate"] == 6
    assert ("restore", 150) in sim.log and ("lb", 150) in sim.log


def test_last_window_is_audited():
    sim = FakeSim([True, True])
    st = S.rollout(sim, None, windows=5, K=50, tip_tol=1.0, audit_every=4, backoff=1, cx=0, cy=0)
    assert sim.source == ["nn", "nn", "nn", "lb", "lb"]
    assert st["audited"] == 2


def test_lb_first_windows():
    sim = FakeSim([True, True])
    st = S.rollout(sim, None, windows=8, K=50, tip_tol=1.0, audit_every=3, backoff=1, cx=0, cy=0, lb_first=2)
    assert sim.source == ["lb", "lb", "nn", "nn", "lb", "nn", "nn", "lb"]
    assert st["lb_first"] == 2 and st["surrogate"] == 4


def test_drift_budget_stops_the_network():
    """Audits pass with 0.15 lattice units each; every one charges 0.15 per
    network window it covers (3): after two audits 0.9 is charged and the
    next stretch would reach 1.35 > 1, so the rest goes to the LB."""
    sim = FakeSim([True] * 10)
    sim.err = 0.15
    st = S.rollout(sim, None, windows=20, K=50, tip_tol=1.0, audit_every=4, backoff=1, cx=0, cy=0)
    assert sim.source[:8] == ["nn", "nn", "nn", "lb"] * 2
    assert sim.source[8:] == ["lb"] * 12 and sim.steps == 1000
    assert abs(st["drift_charged"] - 0.9) < 1e-12 and st["lb_after_budget"] == 12


def test_without_drift_budget_only_window_audits_judge():
    """drift_budget = inf: the per-window reading of the fallback; the same
    passing audits as above never stop the network."""
    sim = FakeSim([True] * 10)
    sim.err = 0.15
    st = S.rollout(sim, None, windows=20, K=50, tip_tol=1.0, audit_every=4, backoff=1, cx=0, cy=0,
                   drift_budget=float("inf"))
    assert sim.source == ["nn", "nn", "nn", "lb"] * 5
    assert st["lb_after_budget"] == 0 and st["surrogate"] == 15
    assert abs(st["drift_charged"] - 0.15 * 15) < 1e-12
