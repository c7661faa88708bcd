"""Split the links of a batch over ranks (one GPU per rank).

Links are independent problems (each is its own DRT run over its own time grid), so a batch shards by
link with no data-path collective: each rank synthesises H for its links only and the job's
throughput is the units of all ranks over the slowest rank's time.  The work of a link is
n_paths x n_steps path-steps (its synthesis scales with n_steps x n_bins on top, the same for every
link of a batch of one bin count).  Greedy longest-processing-time assignment: links in decreasing
order of work, each to the rank with the least work so far (ties to the lower rank), which keeps every
rank's load within the largest single link of the mean.  Host logic only; deterministic, so every rank
computes the same split without communicating.
"""
from __future__ import annotations

import heapq


def partition_links(work, n_ranks: int) -> list[list[int]]:
    """Indices of the links each rank takes, in increasing order; `work` holds each link's cost."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    heap = [(0.0, r) for r in range(n_ranks)]
    out: list[list[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(work[i]), r))
    return [sorted(x) for x in out]


def rank_links(work, rank: int, n_ranks: int) -> list[int]:
    """The links of one rank (see partition_links)."""
    return partition_links(work, n_ranks)[rank]
