"""Partition of independent systems over ranks (the batched form on several GPUs).

Independent systems need no exchange: each rank sets up and solves its own share, and only
per-system results (iterations, status, times) are combined on the host.  The share of a system
is its nonzero count, which the setup and every V-cycle scale with.
"""
from __future__ import annotations


def partition(weights, nparts: int) -> list[list[int]]:
    """Greedy longest-processing-time partition: systems in decreasing weight (ties by index) go to
    the part with the smallest load so far (ties by part index).  Returns, per part, its system
    indices in ascending order.  Deterministic, so every rank computes the same partition.  The
    largest load is at most the average load plus the largest weight."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    w = [float(x) for x in weights]
    if any(x < 0 for x in w):
        raise ValueError("weights must be non-negative")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    load = [0.0] * nparts
    parts: list[list[int]] = [[] for _ in range(nparts)]
    for i in order:
        p = min(range(nparts), key=lambda k: (load[k], k))
        parts[p].append(i)
        load[p] += w[i]
    return [sorted(p) for p in parts]
