"""List chunking and halo plans for running the sparse sweep on P ranks.

The flow solver cuts the 1-D fluid-cell list into P equal chunks (the
first N mod P chunks hold one cell more), so every rank owns the same work;
each rank finds the links whose source cell lives in another chunk
("remote links"), receives those PDFs into ghost cells before every step,
and sweeps its chunk with a local adjacency list (Sec. 2, the flow solver's
domain decomposition; Fig. 1c).  The interface metrics the paper uses to
explain the ordering effect -- neighbour partitions and remote links per
partition (Sec. 7, Fig. 7) -- come out of the same plan.

Local layout of rank k with n_k cells and G_k ghosts: PDF array of
19 * n_k + G_k elements, own PDFs in SoA rows q * n_k + i, ghosts after
them.  Local adjacency entry for a global entry q * N + m: q * n_k + (m - b_k)
if m is in the chunk, else 19 * n_k + g with g the ghost slot of (q, m).
Ghosts are grouped by owner rank (ascending), and inside a group sorted by
the owner's local slot, so a peer's contribution is one contiguous run.

This module is host-side planning on numpy arrays; the exchange itself is
``lbm_halo_gather`` (a device gather by slot list) on the GPU, or any
point-to-point transport between processes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def chunk_bounds(n: int, p: int) -> np.ndarray:
    """begin[0..p] of p chunks of an n-cell list; sizes differ by at most
    one, the larger ones first."""
    if p < 1:
        raise ValueError("need at least one chunk")
    q, r = divmod(int(n), int(p))
    k = np.arange(p + 1, dtype=np.int64)
    return k * q + np.minimum(k, r)


def owner_of(m: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Chunk owning each global cell index."""
    return np.searchsorted(bounds, m, side="right") - 1


@dataclass
class RankPlan:
    rank: int
    begin: int
    count: int
    adj: np.ndarray                 # int32 [18, count] local adjacency
    ghost_owner: np.ndarray         # int32 [G] owning rank of each ghost
    ghost_src: np.ndarray           # int64 [G] owner-local slot of each ghost
    recv_from: dict = field(default_factory=dict)   # peer -> (ghost offset, length)

    @property
    def n_ghost(self) -> int:
        return int(self.ghost_src.size)

    @property
    def local_size(self) -> int:
        return 19 * self.count + self.n_ghost


def plan(adj: np.ndarray, n: int, p: int):
    """Per-rank plans for p chunks of a sparse representation with global
    adjacency ``adj`` [18, n] (flat source slots q * n + m).

    Returns (plans, send): ``send[k][j]`` is the int64 array of rank-k local
    slots that rank k sends to rank j, in the order of j's ghost run."""
    adj = np.asarray(adj, dtype=np.int64).reshape(18, n)
    bounds = chunk_bounds(n, p)
    plans = []
    send = [dict() for _ in range(p)]
    for k in range(p):
        b, e = int(bounds[k]), int(bounds[k + 1])
        nk = e - b
        a = adj[:, b:e]
        q = a // max(n, 1)
        m = a - q * n
        local = (m >= b) & (m < e)
        out = np.empty((18, nk), dtype=np.int64)
        out[local] = q[local] * nk + (m[local] - b)
        rq, rm = q[~local], m[~local]
        own = owner_of(rm, bounds)
        own_slot = rq * (bounds[own + 1] - bounds[own]) + (rm - bounds[own])
        key = own * (19 * (n + 1)) + own_slot
        uniq, inverse = np.unique(key, return_inverse=True)
        g_owner = uniq // (19 * (n + 1))
        g_slot = uniq - g_owner * (19 * (n + 1))
        out[~local] = 19 * nk + inverse
        recv = {}
        for j in np.unique(g_owner):
            idx = np.nonzero(g_owner == j)[0]
            recv[int(j)] = (int(idx[0]), int(idx.size))
            send[int(j)][k] = g_slot[idx].astype(np.int64)
        if 19 * nk + uniq.size >= 2 ** 31:
            raise OverflowError("local PDF array exceeds the int32 slot range")
        plans.append(RankPlan(k, b, nk, out.astype(np.int32), g_owner.astype(np.int32),
                              g_slot.astype(np.int64), recv))
    return plans, send


def interface_metrics(adj: np.ndarray, n: int, p: int):
    """Per-chunk neighbour-partition counts and remote-link counts (the two
    histograms of Fig. 7): a remote link is an adjacency entry whose source
    cell lies in another chunk; its chunk is a neighbour partition."""
    adj = np.asarray(adj, dtype=np.int64).reshape(18, n)
    bounds = chunk_bounds(n, p)
    m = adj % max(n, 1)
    cell_owner = owner_of(np.arange(n), bounds)
    src_owner = owner_of(m, bounds)
    remote = src_owner != cell_owner[None, :]
    links = np.bincount(cell_owner[np.nonzero(remote)[1]], minlength=p)
    pairs = np.unique(np.stack([np.broadcast_to(cell_owner, m.shape)[remote],
                                src_owner[remote]]), axis=1)
    neighbours = np.bincount(pairs[0], minlength=p) if pairs.size else np.zeros(p, np.int64)
    return neighbours.astype(np.int64), links.astype(np.int64)
