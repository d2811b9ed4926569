"""Autotuner host logic without a GPU: per-class choice of the fastest tier
from the plans' launch timings, tiers a class cannot use skipped, and the
JSON round trip -- against fakes of the device calls."""
import sys

import numpy as np

from paper_2605_10312_gb300 import eri, synth, tune


class _Stream:
    def synchronize(self):
        pass


class _Cuda:
    @staticmethod
    def current_stream():
        return _Stream()


class _Torch:
    float64 = "float64"
    cuda = _Cuda()

    @staticmethod
    def empty(n, dtype=None, device=None):
        return np.empty(n)


# microseconds per quartet of each (class, tier); a missing entry: the tier
# cannot run that class
_COST = {(1, 1, 1, 1): {"reg": 2.0, "coop": 3.0, "shared": 5.0, "global": 9.0},
         (2, 2, 2, 2): {"coop": 7.0, "shared": 6.0, "global": 40.0}}


def _fake_plan_class(canon):
    class FakePlan:
        def __init__(self, basis, quartets, tier="auto", **kw):
            self.q = np.asarray(quartets)
            self.cls = canon(basis, self.q)
            if tier not in _COST[self.cls]:
                raise eri.EriError(-2, "tier not built for this class")
            self.tier = tier
            self.output_count = 1

        def set_timing(self, on=True):
            pass

        def compute(self, out, stream=None):
            pass

        def launches(self):
            n = self.q.shape[0]
            # record 0 is the pair set-up; one launch for the class
            return [{"cls": (-1, -1, -1, -1), "tier": 0, "ms": 0.0, "quartets": 0},
                    {"cls": self.cls, "tier": eri.TIERS[self.tier], "quartets": n,
                     "ms": _COST[self.cls][self.tier] * n / 1e3}]

        def close(self):
            pass
    return FakePlan


def test_autotune_picks_the_fastest_feasible_tier(monkeypatch, tmp_path):
    monkeypatch.setitem(sys.modules, "torch", _Torch())

    def canon(basis, q):
        return tuple(int(x) for x in tune._group_key(basis, q[0]))
    monkeypatch.setattr(eri, "Plan", _fake_plan_class(canon))
    applied = {}
    monkeypatch.setattr(eri, "set_class_tier", lambda c, t: applied.__setitem__(tuple(c), t))
    b1, q1 = synth.class_sweep((1, 1, 1, 1), 40, seed=1)
    b2, q2 = synth.class_sweep((2, 2, 2, 2), 30, seed=2)
    basis, q = synth.concat_sets([(b1, q1), (b2, q2)], shuffle_seed=3)
    res = tune.autotune(basis, q, sample=16)
    assert res[(1, 1, 1, 1)]["tier"] == "reg" and res[(2, 2, 2, 2)]["tier"] == "shared"
    assert set(res[(2, 2, 2, 2)]["us_per_quartet"]) == {"coop", "shared", "global"}   # reg skipped
    assert abs(res[(1, 1, 1, 1)]["us_per_quartet"]["coop"] - 3.0) < 1e-12
    assert applied == {(1, 1, 1, 1): "reg", (2, 2, 2, 2): "shared"}
    path = tmp_path / "tiers.json"
    tune.save(res, path)
    applied.clear()
    again = tune.load(path)
    assert again == res and applied == {(1, 1, 1, 1): "reg", (2, 2, 2, 2): "shared"}
