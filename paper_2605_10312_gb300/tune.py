"""Autotuner: per-class tier choice from timed trials.

For every class a workload touches, the quartets of that class group are run
on each feasible tier (compiled register, team-cooperative, shared-memory or
global-scratch program) with launch timing on, and the fastest per quartet
becomes the class's preferred tier in the runtime (eri_set_class_tier).
Results can be saved and reloaded as JSON keyed by class.
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


def autotune(basis, quartets, sample=2048, reps=2, tiers=TIERS, apply=True, seed=0):
    """Time each tier on up to `sample` quartets of every class group; returns
    {class: {"tier": best, "us_per_quartet": {tier: t}}} and, with apply,
    installs the choices in the runtime."""
    import torch
    q = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)
    keys = [_group_key(basis, x) for x in q]
    groups = {}
    for i, k in enumerate(keys):
        groups.setdefault(k, []).append(i)
    rng = np.random.default_rng(seed)
    stream = torch.cuda.current_stream()
    per_cls = {}
    for k, idx in groups.items():
        idx = np.array(idx)
        if idx.size > sample:
            idx = rng.choice(idx, sample, replace=False)
        sub = q[idx]
        for tier in tiers:
            try:
                p = eri.Plan(basis, sub, tier=tier)
            except eri.EriError:
                continue
            out = torch.empty(max(1, p.output_count), dtype=torch.float64, device="cuda")
            p.set_timing(True)
            p.compute(out, stream)  # warm-up (program upload, caches)
            best = {}
            for _ in range(reps):
                p.compute(out, stream)
                stream.synchronize()
                for rec in p.launches()[1:]:
                    c = rec["cls"]
                    key = (c, rec["tier"])
                    t = rec["ms"] * 1e3 / max(1, rec["quartets"])
                    best.setdefault(c, {})
                    best[c][key] = min(best[c].get(key, float("inf")), t)
            for c, d in best.items():
                ent = per_cls.setdefault(c, {})
                for (cc, t_id), t in d.items():
                    name = eri.TIERS_INV[t_id]
                    ent[name] = min(ent.get(name, float("inf")), t)
            p.close()
    result = {}
    for c, d in per_cls.items():
        bt = min(d, key=d.get)
        result[c] = {"tier": bt, "us_per_quartet": d}
        if apply:
            eri.set_class_tier(c, bt)
    return result


def save(result, path):
    with open(path, "w") as f:
        json.dump({"".join(map(str, c)): v for c, v in result.items()}, f, indent=1)


def load(path, apply=True):
    with open(path) as f:
        raw = json.load(f)
    result = {tuple(int(ch) for ch in k): v for k, v in raw.items()}
    if apply:
        for c, v in result.items():
            eri.set_class_tier(c, v["tier"])
    return result
