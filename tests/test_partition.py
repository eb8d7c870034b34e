"""List chunking, halo plans and interface metrics (host logic, CPU).

A chunked step -- every rank pulls through its local adjacency from its
own PDFs plus ghosts filled from the owners -- must reproduce the unsplit
step bit for bit (the per-cell arithmetic is the same)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1111_1129_gb300 import inputs
from paper_1111_1129_gb300.partition import chunk_bounds, interface_metrics, plan

WP = 1.0 / 0.8
WM = oracle.omega_minus(WP)


@pytest.mark.parametrize("n,p", [(10, 3), (7, 7), (100, 8), (5, 1), (3, 5)])
def test_chunks_differ_by_at_most_one(n, p):
    b = chunk_bounds(n, p)
    sizes = np.diff(b)
    assert b[0] == 0 and b[-1] == n
    assert sizes.max() - sizes.min() <= 1
    assert np.all(np.diff(sizes) <= 0)          # the larger chunks first


def test_sparse_step_matches_dense_pull():
    """Pin of the oracle's sparse stepper: one step through the oracle's
    adjacency equals the dense full-array step, bit for bit."""
    rng = np.random.default_rng(1)
    flags = (rng.random((5, 6, 7)) < 0.3).astype(np.uint8)
    cells, _, adj = oracle.build_sparse(flags, oracle.ORDER_MORTON1, periodic=0b101)
    f0 = oracle.rest_state(flags) * (1 + 0.05 * rng.standard_normal((19,) + flags.shape))
    F = [1e-3, -2e-4, 5e-4]
    alpha = 0.05 * rng.random(flags.shape)
    fd, _, _, _ = oracle.run(flags, 0b101, WP, WM, F, 1, alpha=alpha, f=f0)
    fs = oracle.sparse_step(oracle.to_sparse(f0, cells), adj, len(cells), F, WP, WM,
                            alpha=oracle.to_sparse(alpha, cells))
    np.testing.assert_array_equal(fs.reshape(19, -1), oracle.to_sparse(fd, cells))


def _chunked_run(f, adj, n, p, steps, F):
    plans, send = plan(adj, n, p)
    local = []
    for pl in plans:
        own = f.reshape(19, n)[:, pl.begin:pl.begin + pl.count].ravel()
        local.append(np.concatenate([own, np.zeros(pl.n_ghost)]))
    for _ in range(steps):
        for k, pl in enumerate(plans):          # exchange
            for j, (off, length) in pl.recv_from.items():
                s = 19 * pl.count + off
                local[k][s:s + length] = local[j][send[j][k]]
        new = []
        for k, pl in enumerate(plans):          # sweep each chunk
            out = oracle.sparse_step(local[k], pl.adj, pl.count, F, WP, WM)
            new.append(np.concatenate([out, np.zeros(pl.n_ghost)]))
        local = new
    return np.concatenate([local[k][:19 * pl.count].reshape(19, -1)
                           for k, pl in enumerate(plans)], axis=1)


@pytest.mark.parametrize("p", [1, 2, 3, 7])
@pytest.mark.parametrize("ordering", [oracle.ORDER_LEX, oracle.ORDER_BLOCKED, oracle.ORDER_MORTON1])
def test_chunked_steps_equal_the_unsplit_run(p, ordering):
    bed = inputs.packed_bed((14, 12, 16), 2, 11.0, 2.5, 0.45, 9)
    cells, _, adj = oracle.build_sparse(bed.flags, ordering, (4, 4, 4), bed.periodic)
    n = len(cells)
    rng = np.random.default_rng(p)
    f0 = oracle.to_sparse(oracle.rest_state(bed.flags), cells) * (
        1 + 0.01 * rng.standard_normal((19, n)))
    F = [0.0, 0.0, 1e-4]
    ref = f0.ravel()
    for _ in range(4):
        ref = oracle.sparse_step(ref, adj, n, F, WP, WM)
    got = _chunked_run(f0.ravel(), adj, n, p, 4, F)
    np.testing.assert_array_equal(got, ref.reshape(19, n))


def test_local_adjacency_reads_the_same_values():
    bed = inputs.bed_small(0)
    cells, _, adj = oracle.build_sparse(bed.flags, oracle.ORDER_LEX, periodic=bed.periodic)
    n = len(cells)
    f = np.random.default_rng(0).random(19 * n)
    plans, send = plan(adj, n, 5)
    for k, pl in enumerate(plans):
        arr = np.concatenate([f.reshape(19, n)[:, pl.begin:pl.begin + pl.count].ravel(),
                              np.zeros(pl.n_ghost)])
        for j, (off, length) in pl.recv_from.items():
            peer = plans[j]
            peer_arr = f.reshape(19, n)[:, peer.begin:peer.begin + peer.count].ravel()
            arr[19 * pl.count + off:19 * pl.count + off + length] = peer_arr[send[j][k]]
        np.testing.assert_array_equal(arr[pl.adj], f[adj[:, pl.begin:pl.begin + pl.count]])


def test_interface_metrics_brute_force():
    rng = np.random.default_rng(3)
    flags = (rng.random((6, 5, 4)) < 0.3).astype(np.uint8)
    cells, _, adj = oracle.build_sparse(flags, oracle.ORDER_LEX, periodic=0b111)
    n, p = len(cells), 4
    nb, links = interface_metrics(adj, n, p)
    b = chunk_bounds(n, p)
    own = lambda c: int(np.searchsorted(b, c, side="right") - 1)
    ref_links = [0] * p
    ref_nb = [set() for _ in range(p)]
    for i, c in itertools.product(range(18), range(n)):
        m = int(adj[i, c]) % n
        if own(m) != own(c):
            ref_links[own(c)] += 1
            ref_nb[own(c)].add(own(m))
    assert list(links) == ref_links
    assert list(nb) == [len(s) for s in ref_nb]


def test_blocking_trades_neighbours_for_fewer_remote_links():
    """Lexicographic order cuts the domain into slices (few neighbour
    partitions, many remote links); blocking makes more neighbour
    partitions but fewer remote links (Sec. 7, Fig. 7)."""
    bed = inputs.packed_bed((48, 48, 96), 2, 46.0, 4.0, 0.45, 1)
    out = {}
    for name, kind, block in [("lex", oracle.ORDER_LEX, (1, 1, 1)),
                              ("blocked16", oracle.ORDER_BLOCKED, (16, 16, 16))]:
        cells, _, adj = oracle.build_sparse(bed.flags, kind, block, bed.periodic)
        nb, links = interface_metrics(adj, len(cells), 32)
        out[name] = (nb.mean(), links.mean())
    assert out["lex"][0] < out["blocked16"][0]
    assert out["lex"][1] > out["blocked16"][1]
