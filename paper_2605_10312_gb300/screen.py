"""Schwarz screening on the device (the batched mixed-class workload).

The Schwarz factor of a shell pair, Q_ab = sqrt(max |(ab|ab)|), is computed
from the pair's own diagonal block, evaluated by the ERI kernels, and reduced
on the device (eri_schwarz); quartets with Q_ab Q_cd below the threshold are
dropped (|(ab|cd)| <= Q_ab Q_cd).
"""
from __future__ import annotations

import numpy as np

from . import eri, synth


def pair_bounds_device(basis, pairs=None, stream=None):
    """(pairs [npair, 2] host int32, Q [npair] CUDA float64 tensor) for every
    unique shell pair (a >= b); Q stays on the device."""
    import torch
    if pairs is None:
        pairs = synth.shell_pairs(basis.nshell)
    diag = np.ascontiguousarray(np.concatenate([pairs, pairs], axis=1).astype(np.int32))
    p = eri.Plan(basis, diag)
    blocks = torch.empty(max(1, p.output_count), dtype=torch.float64, device="cuda")
    bounds = torch.empty(max(1, diag.shape[0]), dtype=torch.float64, device="cuda")
    p.compute(blocks, stream)
    p.schwarz(blocks, bounds, stream)
    p.close()
    return pairs, bounds[: diag.shape[0]]


def pair_bounds(basis, pairs=None, stream=None):
    """(pairs [npair, 2], Q [npair]) for every unique shell pair (a >= b)."""
    pairs, q = pair_bounds_device(basis, pairs, stream)
    return pairs, q.cpu().numpy()


def screened(basis, threshold=1e-10, stream=None):
    """Unique quartets of the basis surviving Schwarz screening, [n, 4]
    (host enumeration of the device bounds)."""
    pairs, q = pair_bounds(basis, stream=stream)
    return synth.screened_quartets(q, pairs, threshold)


def screened_device(basis, threshold=1e-10, stream=None):
    """The same survivors listed on the device (eri_screen_quartets: a
    counting pass, a prefix sum and a compaction over the device bounds);
    a CUDA int32 tensor [n, 4].  The pairs go in sorted by falling bound
    (stably), so the list comes out in the host enumeration's order and
    orientation, element for element: screened quartets of one pair of
    small bound together, which keeps the J/K digestion's reads and
    reductions of neighbouring quartets on shared L2 lines."""
    import torch
    pairs, q = pair_bounds_device(basis, stream=stream)
    dp = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).to(q.device)
    qs, ps = sort_pairs(q, dp)
    return eri.screen_quartets(qs, ps, threshold, stream)


def sort_pairs(q, pairs):
    """Pair factors (CUDA float64 [npair]) and pairs (CUDA int32 [npair, 2])
    reordered by falling factor, ties in index order, on the device."""
    import torch
    order = torch.argsort(-q, stable=True)
    return q[order].contiguous(), pairs[order].contiguous()


def quartet_bounds(pair_q, quartets):
    """Schwarz bound Q_ab Q_cd of each quartet, given the per-pair factors of
    synth.shell_pairs order (pair (a, b), a >= b, at a (a + 1) / 2 + b)."""
    q = np.asarray(quartets, dtype=np.int64).reshape(-1, 4)

    def idx(a, b):
        hi, lo = np.maximum(a, b), np.minimum(a, b)
        return hi * (hi + 1) // 2 + lo
    return pair_q[idx(q[:, 0], q[:, 1])] * pair_q[idx(q[:, 2], q[:, 3])]
