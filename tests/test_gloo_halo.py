"""The chunked path with real processes: two gloo ranks on the CPU, each
owning one chunk of the list, exchanging ghost PDFs with point-to-point
messages before every step and stepping their chunk with the CPU oracle's
sparse stepper.  The gathered result must equal the unsplit run bit for
bit; a rank that raises is reported on the host, no GPU involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

WP = 1.0 / 0.8
STEPS = 5
F = (0.0, 0.0, 1e-4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import oracle
    from paper_1111_1129_gb300 import inputs
    bed = inputs.packed_bed((14, 12, 16), 2, 11.0, 2.5, 0.45, 9)
    cells, _, adj = oracle.build_sparse(bed.flags, oracle.ORDER_BLOCKED, (4, 4, 4), bed.periodic)
    n = len(cells)
    f0 = oracle.to_sparse(oracle.rest_state(bed.flags), cells) * (
        1 + 0.01 * np.random.default_rng(0).standard_normal((19, n)))
    return adj, n, f0.ravel()


def _worker(rank, world, port, out_dir, fail_rank):
    import oracle
    from paper_1111_1129_gb300.partition import plan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError(f"rank {rank} failed on purpose before its first exchange")
        adj, n, f0 = _problem()
        plans, send = plan(adj, n, world)
        me = plans[rank]
        wm = oracle.omega_minus(WP)
        own = f0.reshape(19, n)[:, me.begin:me.begin + me.count].ravel()
        local = np.concatenate([own, np.zeros(me.n_ghost)])
        for _ in range(STEPS):
            reqs = []
            for j, slots in send[rank].items():
                reqs.append(dist.isend(torch.from_numpy(local[slots].copy()), dst=j))
            for j, (off, length) in sorted(me.recv_from.items()):
                buf = torch.empty(length, dtype=torch.float64)
                dist.recv(buf, src=j)
                s = 19 * me.count + off
                local[s:s + length] = buf.numpy()
            for r in reqs:
                r.wait()
            out = oracle.sparse_step(local, me.adj, me.count, F, WP, wm)
            local = np.concatenate([out, np.zeros(me.n_ghost)])
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), local[:19 * me.count])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsplit_run(tmp_path):
    import oracle
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), -1), nprocs=world, join=True)
    adj, n, f0 = _problem()
    ref = f0
    for _ in range(STEPS):
        ref = oracle.sparse_step(ref, adj, n, F, WP, oracle.omega_minus(WP))
    from paper_1111_1129_gb300.partition import chunk_bounds
    b = chunk_bounds(n, world)
    parts = [np.load(tmp_path / f"rank{k}.npy").reshape(19, -1) for k in range(world)]
    for k in range(world):
        assert parts[k].shape[1] == b[k + 1] - b[k]
    np.testing.assert_array_equal(np.concatenate(parts, axis=1), ref.reshape(19, n))


def test_a_failing_rank_is_reported_on_the_host(tmp_path):
    """Rank 1 raises before its first exchange; whichever the host learns of
    first -- rank 1's error or rank 0's broken connection -- ends the job
    with an error instead of a hang."""
    with pytest.raises(Exception) as ei:
        mp.spawn(_worker, args=(2, _free_port(), str(tmp_path), 1), nprocs=2, join=True)
    msg = str(ei.value)
    assert "failed on purpose" in msg or "Connection closed" in msg or "Connection reset" in msg
