"""One M-RA problem sharded over the ranks of a process group (Sec. 3.5).

The regions of one resolution are independent, so the level-s subtrees of a
streamed handle (stream_level = s) are split into contiguous ranges, one per
rank.  Every rank builds the same handle (the data are replicated), evaluates
its own subtrees (``loglik_subtrees``), the ranks exchange the subtrees'
summaries in one all-gather, and every rank finishes the coarse levels s..0
(``loglik_combine``) with the same result.  The exchange is the only
collective; it moves nsub x len doubles (about 3 MB at s = 2, r = 64).

``evaluator`` is anything with ``summary_len()``, ``loglik_subtrees(theta,
first, count)`` and ``loglik_combine(theta, summaries)``: a GPU handle
(paper_1507_04789_gb300.mra.Handle), or any object with that interface.
"""
from __future__ import annotations

import numpy as np


def subtree_range(nsub: int, rank: int, world: int):
    """Contiguous block of level-s subtrees of ``rank``: (first, count)."""
    q, rem = divmod(nsub, world)
    first = rank * q + min(rank, rem)
    return first, q + (1 if rank < rem else 0)


def all_gather_rows(local: np.ndarray, nsub: int, world: int, group=None, device=None) -> np.ndarray:
    """All-gather of every rank's summary rows (in rank order, so in subtree
    order) into one (nsub x len) array, through torch.distributed."""
    import torch
    import torch.distributed as dist
    cplx = np.iscomplexobj(local)
    if cplx:                                   # complex rows travel as (re, im) pairs
        local = np.ascontiguousarray(local, dtype=np.complex128).view(np.float64)
    length = local.shape[1]
    counts = [subtree_range(nsub, k, world)[1] for k in range(world)]
    width = max(counts)
    buf = torch.zeros((width, length), dtype=torch.float64, device=device)
    if local.shape[0]:
        buf[: local.shape[0]] = torch.from_numpy(np.ascontiguousarray(local)).to(device)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    rows = np.concatenate([parts[k][: counts[k]].cpu().numpy() for k in range(world)], axis=0)
    return rows.view(np.complex128) if cplx else rows


def sharded_loglik(evaluator, theta, rank: int, world: int, group=None, device=None) -> float:
    """The log-likelihood of the whole problem, with this rank's share of the
    level-s subtrees evaluated here; every rank returns the same value."""
    length, nsub = evaluator.summary_len()
    first, count = subtree_range(nsub, rank, world)
    local = evaluator.loglik_subtrees(theta, first, count)
    if world > 1:
        summaries = all_gather_rows(local, nsub, world, group, device)
    else:
        summaries = local
    return evaluator.loglik_combine(theta, summaries)
