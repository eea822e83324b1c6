"""Host logic of the surrogate rollout policy (audit every A windows, restore
and re-run by the LB on a failed audit, back-off), against a fake solver that
records what it is asked to do."""
from __future__ import annotations

from paper_2209_01444_gb300 import lbm as L
from paper_2209_01444_gb300 import surrogate as S


class FakeSim:
    """Tracks the step count and which windows the state came from."""

    def __init__(self, verdicts, nonfinite=(), raises=()):
        self.steps = 0
        self.source = []      # per window: "nn" or "lb"
        self.snap = None
        self.verdicts = list(verdicts)  # accepted flags of successive audits
        self.nonfinite = set(nonfinite)  # unaudited calls (0, 1, ...) whose prediction is not finite
        self.raises = set(raises)  # audits (0, 1, ...) whose LB run goes non-finite
        self.audits = 0
        self.calls = 0
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
        if not audit:
            call, self.calls = self.calls, self.calls + 1
            if call in self.nonfinite:  # not applied: the state stays where it was
                self.log.append(("nonfinite", self.steps))
                return {"audited": False, "accepted": False, "tip_err": float("inf")}
            self.steps += K
            self.source.append("nn")
            return {"audited": False, "accepted": True, "tip_err": 0.0}
        audit_no, self.audits = self.audits, self.audits + 1
        self.steps += K
        self.source.append("lb")  # an audited window keeps the LB result
        if audit_no in self.raises:
            raise L.LBMError(L.LBM_ENUMERIC, "non-finite value in the state")
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


def test_nonfinite_prediction_is_not_kept_and_the_stretch_rerun():
    """An unaudited window whose prediction is not finite leaves the state
    unchanged; the policy treats it as a failed audit: back to the last
    audited snapshot, the LB re-runs the network windows since then and this
    window, and the network sits out the back-off."""
    sim = FakeSim([True, True, True], nonfinite={3})
    st = S.rollout(sim, None, windows=12, K=50, tip_tol=1.0, audit_every=3, backoff=2, cx=0, cy=0)
    assert sim.steps == 600
    # windows 0-1 nn, 2 audited; window 3 nn; window 4's prediction is not finite:
    # 3-4 re-run by the LB; 5-6 back off; 7-8 nn, 9 audited; 10 nn, 11 audited (last)
    assert sim.source == ["nn", "nn", "lb"] + ["lb", "lb"] + ["lb", "lb"] + ["nn", "nn", "lb"] + ["nn", "lb"]
    assert st["rejected"] == 1 and st["nonfinite"] == 1 and st["lb_rerun"] == 1 and st["lb_backoff"] == 2
    assert st["surrogate"] == 5
    assert ("nonfinite", 200) in sim.log and ("restore", 150) in sim.log


def test_audit_that_goes_nonfinite_is_a_failed_audit():
    """The LB run of an audit goes non-finite (the network windows before it
    kept a finite but unphysical state): the policy restores the last passed
    audit's snapshot, the LB re-runs the stretch, and the network backs off."""
    sim = FakeSim([True, True, True], raises={1})
    st = S.rollout(sim, None, windows=12, K=50, tip_tol=1.0, audit_every=3, backoff=2, cx=0, cy=0)
    assert sim.steps == 600
    # 0-1 nn, 2 audited; 3-4 nn, the audit of 5 raises: 3-5 re-run by the LB;
    # 6-7 back off; 8-9 nn, 10 audited; 11 audited (last)
    assert sim.source == ["nn", "nn", "lb"] + ["lb"] * 3 + ["lb"] * 2 + ["nn", "nn", "lb"] + ["lb"]
    assert st["rejected"] == 1 and st["nonfinite"] == 1 and st["lb_rerun"] == 2 and st["lb_backoff"] == 2
    assert st["surrogate"] == 4


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
