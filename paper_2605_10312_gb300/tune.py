"""Autotuner: per-class tier choice, and per-(class, kind of contraction)
cooperative shape and vote form, from timed trials.

For every class a workload touches, the quartets of that class group are run
on each feasible tier (compiled register, team-cooperative, shared-memory or
global-scratch program) with launch timing on, and the fastest per quartet
becomes the class's preferred tier in the runtime (eri_set_class_tier).
For the classes that then run on the team-cooperative tier, every shape the
build ships (eri_class_shapes: team size, nodes per lane, steps per wave of
each phase) is timed with the optional FP64 terms predicated and behind warp
votes, separately for deep, shallow and single-primitive parts (the launch
records say which), and the fastest per kind is installed
(eri_set_class_shape).  Results can be saved and reloaded as JSON keyed by
class.
"""
from __future__ import annotations

import json

import numpy as np

from . import eri

TIERS = ("reg", "coop", "shared", "global")


def _group_key(basis, q):
    l = basis.shell_l[q]
    a = (max(l[0], l[1]), min(l[0], l[1]))
    b = (max(l[2], l[3]), min(l[2], l[3]))
    return a + b if a >= b else b + a


def _samples(basis, quartets, sample, seed):
    q = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)
    keys = [_group_key(basis, x) for x in q]
    groups = {}
    for i, k in enumerate(keys):
        groups.setdefault(k, []).append(i)
    rng = np.random.default_rng(seed)
    out = {}
    for k, idx in groups.items():
        idx = np.array(idx)
        if idx.size > sample:
            idx = rng.choice(idx, sample, replace=False)
        out[k] = q[idx]
    return out


FILL_QUARTETS = 32768   # a trial evaluates at least this many quartets (the sample is repeated) ...
FILL_MS = 200.0         # ... unless that would take longer than this
BIG_MS = 20.0           # a sample whose plan already runs this long is used as it is


def _filled(basis, sub, stream):
    """The sample repeated until a trial measures throughput: a few hundred
    quartets leave most SMs idle, and small plans are bound by the latency
    of their deepest quartets (a 512-quartet (pp|pp) sample ran 3.7 ms, 40
    times its share of the full sweep, on the register tier, whose lanes
    walk a deep contraction serially).  At least FILL_QUARTETS quartets, as
    long as the trial stays within about FILL_MS."""
    import torch
    p = eri.Plan(basis, sub)
    out = torch.empty(max(1, p.output_count), dtype=torch.float64, device="cuda")
    p.set_timing(True)
    p.compute(out, stream)
    p.compute(out, stream)
    stream.synchronize()
    ms = sum(max(0.0, r["ms"]) for r in p.launches())
    p.close()
    if ms >= BIG_MS:
        return sub
    rep = int(max(1, min(np.ceil(FILL_QUARTETS / max(1, sub.shape[0])), np.floor(FILL_MS / max(ms, 1e-3)))))
    return np.ascontiguousarray(np.tile(sub, (rep, 1))) if rep > 1 else sub


def _timed(plan, out, stream, reps, by_kind=True):
    """{(class, tier, kind): (milliseconds, parts)} -- the time of all of a
    key's launches in one run (a class has one launch per part round and
    contraction group) and their quartet parts, the best of reps runs after
    a warm-up (launch timing on).  by_kind False: kind None, all of a class's
    launches on one tier together."""
    plan.set_timing(True)
    plan.compute(out, stream)  # warm-up (program upload, caches)
    best = {}
    for _ in range(reps):
        plan.compute(out, stream)
        stream.synchronize()
        tot = {}
        for rec in plan.launches()[1:]:
            key = (rec["cls"], rec["tier"], rec.get("kind") if by_kind else None)
            ms, n = tot.get(key, (0.0, 0))
            tot[key] = (ms + rec["ms"], n + rec["quartets"])
        for key, v in tot.items():
            if key not in best or v[0] < best[key][0]:
                best[key] = v
    return best


MARGIN = 0.05   # a choice other than the static one must be this much faster in its trial


def _pick(times, static):
    """The fastest entry of {choice: time}, unless the static choice is within
    MARGIN of it: in a batched plan the classes share the GPU, and a trial
    of one class group alone does not see that."""
    best = min(times, key=times.get)
    if static in times and times[best] > (1.0 - MARGIN) * times[static]:
        return static
    return best


def autotune(basis, quartets, sample=2048, reps=2, tiers=TIERS, apply=True, seed=0, shapes=False):
    """Time each tier on up to `sample` quartets of every class group; returns
    {class: {"tier": best, "us_per_quartet": {tier: t}}} and, with apply,
    installs the choices in the runtime.  shapes: then tune the cooperative
    shapes of the classes whose best tier is the cooperative one
    (autotune_shapes; their entries gain "shapes")."""
    import torch
    stream = torch.cuda.current_stream()
    per_cls, static = {}, {}
    subs = _samples(basis, quartets, sample, seed)
    for k, sub in subs.items():
        sub = _filled(basis, sub, stream)
        p = eri.Plan(basis, sub)
        out = torch.empty(max(1, p.output_count), dtype=torch.float64, device="cuda")
        for (c, t_id, _) in _timed(p, out, stream, 1, by_kind=False):
            static.setdefault(c, eri.TIERS_INV[t_id])
        p.close()
        for tier in tiers:
            try:
                p = eri.Plan(basis, sub, tier=tier)
            except eri.EriError:
                continue
            out = torch.empty(max(1, p.output_count), dtype=torch.float64, device="cuda")
            # tiers cut a class into different parts (the cooperative tier
            # chunks deep contractions), so they compare by the whole
            # class's time on the same sample, per sample quartet
            for (c, t_id, _), (ms, _) in _timed(p, out, stream, reps, by_kind=False).items():
                ent = per_cls.setdefault(c, {})
                name = eri.TIERS_INV[t_id]
                ent[name] = min(ent.get(name, float("inf")), ms * 1e3 / max(1, sub.shape[0]))
            p.close()
    result = {}
    for c, d in per_cls.items():
        bt = _pick(d, static.get(c))
        result[c] = {"tier": bt, "static": static.get(c), "us_per_quartet": d}
        if apply:
            eri.set_class_tier(c, bt)
    if shapes:
        coop_cls = {c for c, v in result.items() if v["tier"] == "coop"}
        found = autotune_shapes(basis, quartets, sample=sample, reps=reps, apply=apply, seed=seed,
                                classes=coop_cls)
        for c, v in found.items():
            result.setdefault(c, {"tier": "coop", "us_per_quartet": {}})["shapes"] = v
    return result


def autotune_shapes(basis, quartets, sample=2048, reps=2, apply=True, seed=0, classes=None):
    """Per class on the cooperative tier (all of them, or those in
    ``classes``) and per kind of contraction present: time every shipped
    shape with both vote forms and keep the fastest.  Returns {class: {kind:
    {"shape": index, "T", "ilp", "k1", "k2": the shape, "votes": "off"|"on",
    "us_per_quartet": {"<index>/<votes>": t}}}}; with apply the choices are
    installed (eri_set_class_shape)."""
    import torch
    stream = torch.cuda.current_stream()
    result = {}
    for _, sub in _samples(basis, quartets, sample, seed).items():
        sub = _filled(basis, sub, stream)
        base = eri.Plan(basis, sub)
        out = torch.empty(max(1, base.output_count), dtype=torch.float64, device="cuda")
        t0 = _timed(base, out, stream, 1)
        default = {(r["cls"], r.get("kind")): "{}/{}".format(r.get("shape"), r.get("votes"))
                   for r in base.launches()[1:] if r["tier"] == eri.TIERS["coop"]}
        base.close()
        present = {}
        for (c, tier, kind) in t0:
            if tier == eri.TIERS["coop"] and kind is not None and (classes is None or c in classes):
                present.setdefault(c, set()).add(kind)
        for c, kinds in present.items():
            cands = eri.class_shapes(c)
            times = {}
            for i in range(len(cands)):
                for votes in ("off", "on"):
                    for kind in eri.KINDS:
                        eri.set_class_shape(c, kind, i, votes)
                    try:
                        p = eri.Plan(basis, sub)
                    except eri.EriError:
                        continue
                    finally:
                        for kind in eri.KINDS:
                            eri.set_class_shape(c, kind, -1)
                    # shapes and vote forms cut the same parts: per part
                    for (cc, tier, kind), (ms, n) in _timed(p, out, stream, reps).items():
                        if cc == c and tier == eri.TIERS["coop"] and kind in kinds:
                            times.setdefault(kind, {})["{}/{}".format(i, votes)] = ms * 1e3 / max(1, n)
                    p.close()
            ent = result.setdefault(c, {})
            for kind, d in times.items():
                best = _pick(d, default.get((c, kind)))
                i, votes = best.split("/")
                ent[kind] = dict(shape=int(i), votes=votes, static=default.get((c, kind)), us_per_quartet=d,
                                 **cands[int(i)])
                if apply:
                    eri.set_class_shape(c, kind, int(i), votes)
    return result


def save(result, path):
    with open(path, "w") as f:
        json.dump({"".join(map(str, c)): v for c, v in result.items()}, f, indent=1)


def load(path, apply=True):
    """Read a saved result; with apply, install its tiers and its shapes (a
    shape is found again by its team size, nodes per lane and wave steps
    among the shapes this build ships; one no longer shipped is skipped)."""
    with open(path) as f:
        raw = json.load(f)
    result = {tuple(int(ch) for ch in k): v for k, v in raw.items()}
    if apply:
        for c, v in result.items():
            eri.set_class_tier(c, v["tier"])
            if v.get("shapes"):
                cands = [tuple(s[k] for k in ("T", "ilp", "k1", "k2")) for s in eri.class_shapes(c)]
                for kind, e in v["shapes"].items():
                    key = tuple(e[k] for k in ("T", "ilp", "k1", "k2"))
                    if key in cands:
                        eri.set_class_shape(c, kind, cands.index(key), e["votes"])
    return result
