"""Host-side partition of independent work units (ensemble members) over
ranks, one GPU per rank.  Members never exchange data, so a multi-GPU run
needs no collective on the data path: each rank advances its own members.
"""
from __future__ import annotations


def member_weight(n_cells: int, n_fine: int, M: int) -> int:
    """Right-hand-side cell evaluations of one LTS3 coarse step, about
    3 nC + 3 M nF (every cell is evaluated in Steps 1, 2 and 4 or 5, the fine
    cells 3 M times in Step 3)."""
    return 3 * int(n_cells) + 3 * int(M) * int(n_fine)


def greedy_partition(weights, parts: int):
    """Longest-processing-time-first: members in decreasing weight (ties by
    index) each go to the currently lightest part (ties: lowest part).
    Deterministic, so every rank computes the same partition.  Returns one
    sorted list of member indices per part."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0] * parts
    out = [[] for _ in range(parts)]
    for i in order:
        p = min(range(parts), key=lambda k: (load[k], k))
        out[p].append(i)
        load[p] += weights[i]
    return [sorted(x) for x in out]
