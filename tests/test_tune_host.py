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
            if tier == "auto":   # the static choice: the first feasible tier
                tier = next(iter(_COST[self.cls]))
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


# microseconds per part of each (class, kind, shape index, votes) on the
# cooperative tier: (dd|dd) deep parts run fastest on shape 1 with votes,
# single-primitive parts on shape 2 without; (ff|ff) keeps shape 0
_SHAPES = {(2, 2, 2, 2): [dict(T=64, ilp=2, k1=1, k2=2, nslot=1104), dict(T=128, ilp=2, k1=1, k2=1, nslot=1500),
                          dict(T=32, ilp=2, k1=1, k2=4, nslot=900)],
           (3, 3, 3, 3): [dict(T=128, ilp=2, k1=1, k2=4, nslot=5146)]}


def _shape_cost(cls, kind, shape, votes):
    if cls == (2, 2, 2, 2):
        if kind == "deep":
            return {0: 5.0, 1: 4.0, 2: 6.0}[shape] - (0.5 if votes == "on" else 0.0)
        return {0: 3.0, 1: 3.5, 2: 2.0}[shape] + (0.25 if votes == "on" else 0.0)
    return 9.0 - (1.0 if votes == "on" else 0.0)


def test_autotune_shapes_picks_per_kind(monkeypatch, tmp_path):
    """Every shipped shape is timed under both vote forms per kind of
    contraction; the fastest per (class, kind) is installed, the trial
    settings are cleared after each plan, and a saved result loads back
    onto the same shape indices."""
    monkeypatch.setitem(sys.modules, "torch", _Torch())
    table = {}                     # the runtime's (class, kind) -> (shape, votes)

    def set_class_shape(ls, kind, shape, votes="auto"):
        if shape < 0:
            table.pop((tuple(ls), kind), None)
        else:
            table[(tuple(ls), kind)] = (shape, votes)

    class FakePlan:
        def __init__(self, basis, quartets, **kw):
            self.q = np.asarray(quartets)
            self.cls = tuple(int(x) for x in tune._group_key(basis, self.q[0]))
            self.output_count = 1
            # a plan freezes the table's entries when it is built
            self.choice = {k: table.get((self.cls, k), (0, "off" if self.cls == (2, 2, 2, 2) else "on"))
                           for k in ("deep", "single")}

        def set_timing(self, on=True):
            pass

        def compute(self, out, stream=None):
            pass

        def launches(self):
            n = self.q.shape[0]
            recs = [{"cls": (-1, -1, -1, -1), "tier": 0, "ms": 0.0, "quartets": 0, "kind": None}]
            for kind, share in (("deep", 3), ("single", 1)):
                s, v = self.choice[kind]
                m = n * share // 4
                recs.append({"cls": self.cls, "tier": eri.TIERS["coop"], "quartets": m, "kind": kind,
                             "ms": _shape_cost(self.cls, kind, s, v) * m / 1e3})
            return recs

        def close(self):
            pass

    monkeypatch.setattr(eri, "Plan", FakePlan)
    monkeypatch.setattr(eri, "class_shapes", lambda ls: [dict(s) for s in _SHAPES[tuple(ls)]])
    monkeypatch.setattr(eri, "set_class_shape", set_class_shape)
    b1, q1 = synth.class_sweep((2, 2, 2, 2), 40, seed=1)
    b2, q2 = synth.class_sweep((3, 3, 3, 3), 40, seed=2)
    basis, q = synth.concat_sets([(b1, q1), (b2, q2)], shuffle_seed=3)
    res = tune.autotune_shapes(basis, q, sample=32)
    dd, ff = res[(2, 2, 2, 2)], res[(3, 3, 3, 3)]
    assert (dd["deep"]["shape"], dd["deep"]["votes"], dd["deep"]["T"]) == (1, "on", 128)
    assert (dd["single"]["shape"], dd["single"]["votes"], dd["single"]["T"]) == (2, "off", 32)
    assert (ff["deep"]["shape"], ff["deep"]["votes"]) == (0, "on")
    assert len(dd["deep"]["us_per_quartet"]) == 6 and len(ff["deep"]["us_per_quartet"]) == 2
    assert table == {((2, 2, 2, 2), "deep"): (1, "on"), ((2, 2, 2, 2), "single"): (2, "off"),
                     ((3, 3, 3, 3), "deep"): (0, "on"), ((3, 3, 3, 3), "single"): (0, "on")}
    path = tmp_path / "shapes.json"
    tune.save({c: {"tier": "coop", "us_per_quartet": {}, "shapes": v} for c, v in res.items()}, path)
    monkeypatch.setattr(eri, "set_class_tier", lambda c, t: None)
    table.clear()
    tune.load(path)
    assert table[((2, 2, 2, 2), "deep")] == (1, "on") and table[((2, 2, 2, 2), "single")] == (2, "off")


def test_pick_keeps_the_static_choice_within_the_margin():
    """A trial winner replaces the static choice only when it is more than
    MARGIN faster; an unknown static choice leaves the fastest."""
    t = {"reg": 1.0, "coop": 0.97}
    assert tune._pick(t, "reg") == "reg"
    assert tune._pick({"reg": 1.0, "coop": 0.90}, "reg") == "coop"
    assert tune._pick(t, None) == "coop" and tune._pick(t, "shared") == "coop"
