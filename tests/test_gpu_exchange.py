"""The chunked path across processes: P ranks (processes sharing one GPU),
each owning one equal chunk of the fluid-cell list, exchange ghost PDFs with
the library's ChunkRunner (lbm_halo_gather packs, torch.distributed point-
to-point messages over gloo through pinned host buffers, then the chunk is
stepped by lbm_step_f64_noalloc on its local adjacency) before every step
(Sec. 2 and Fig. 1c).

The gathered PDFs must equal the FP64 oracle's run of the unsplit bed within
the FP64 tolerance, and the unsplit GPU run (lbm_step on an FP64 state) bit
for bit, with and without Brinkman damping; the all-reduced mass and flux
must match both.  A rank that fails between steps is reported on the host.
No kernel waits on another rank: the ranks meet only on the host, in gloo.
"""
import datetime
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
STEPS = 7
F = (2e-6, -1e-6, 1e-5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bed():
    from paper_1111_1129_gb300 import inputs
    return inputs.packed_bed((20, 18, 24), 2, 17.0, 3.0, 0.45, 11)


def _worker(rank, world, port, out_dir, ordering, fail_rank, damped=False):
    import torch.distributed as dist

    from paper_1111_1129_gb300 import SparseLattice, build, capi, omega_minus
    from paper_1111_1129_gb300.exchange import ChunkRunner
    from paper_1111_1129_gb300.partition import plan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        build.build()
        capi.load()
        bed = _bed()
        lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), ordering, (4, 4, 4), bed.periodic)
        plans, send = plan(lat.adjacency().cpu().numpy(), lat.n, world)
        runner = ChunkRunner(plans[rank], send[rank])
        wm = omega_minus(WP)
        alpha = None
        if damped:   # the rank's own cells of the seeded per-box-cell field
            from paper_1111_1129_gb300 import inputs
            a_box = inputs.alpha_field(bed.dims, seed=4).reshape(-1)
            cells = lat.cells().cpu().numpy()
            me = plans[rank]
            alpha = torch.from_numpy(a_box[cells[me.begin:me.begin + me.count]].copy()).cuda()
        runner.step(3, WP, wm, F, alpha)
        if rank == fail_rank:
            torch.cuda.synchronize()     # nothing of this rank in flight
            raise RuntimeError(f"rank {rank} failed on purpose between steps")
        runner.step(STEPS - 3, WP, wm, F, alpha)
        sums = [runner.reduce_flux(axis, lat.n) for axis in range(3)]
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), runner.pdfs().cpu().numpy())
        if rank == 0:
            np.save(os.path.join(out_dir, "sums.npy"), np.array(sums))
        lat.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ordering,damped", [(2, "lex", False), (3, "blocked", False),
                                                   (2, "blocked", True)])
def test_ranks_reproduce_the_unsplit_run(tmp_path, world, ordering, damped):
    import fp64_measures
    import oracle
    from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, omega_minus
    from paper_1111_1129_gb300.partition import chunk_bounds
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), ordering, -1, damped),
             nprocs=world, join=True)
    build.build()
    capi.load()
    bed = _bed()
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), ordering, (4, 4, 4), bed.periodic)
    n = lat.n
    b = chunk_bounds(n, world)
    parts = [np.load(tmp_path / f"rank{k}.npy") for k in range(world)]
    for k in range(world):
        assert parts[k].shape == (19, b[k + 1] - b[k])
    got = np.concatenate(parts, axis=1)
    sums = np.load(tmp_path / "sums.npy")
    # the oracle's dense run of the unsplit bed
    kind = {"lex": oracle.ORDER_LEX, "blocked": oracle.ORDER_BLOCKED}[ordering]
    cells, _, _ = oracle.build_sparse(bed.flags, kind, (4, 4, 4), bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    a_box = None
    if damped:
        from paper_1111_1129_gb300 import inputs
        a_box = inputs.alpha_field(bed.dims, seed=4)
    f_ref, obs, _, _ = oracle.run(bed.flags, bed.periodic, WP, omega_minus(WP), F, STEPS,
                                  alpha=a_box)
    m = fp64_measures.check(got, oracle.to_sparse(f_ref, cells), STEPS,
                            label=f"exchange {world} ranks {ordering} damped={damped}")
    assert abs(sums[0][0] - obs[-1, 0]) <= 1e-12 * obs[-1, 0]
    for axis in range(3):
        assert abs(sums[axis][1] - obs[-1, 1 + axis] / n) <= 11 * m["bound_abs_df"] + 2.0 ** -61
    # the unsplit GPU run, bit for bit
    st = LBMState(lat, "f64")
    if damped:
        st.set_damping(torch.from_numpy(a_box.reshape(-1)[cells].copy()))
    st.step(STEPS, WP, omega_minus(WP), F)
    np.testing.assert_array_equal(got, st.get_pdfs().cpu().numpy())
    for axis in range(3):
        mass, flux = st.reduce_flux(axis)
        assert abs(sums[axis][0] - mass) <= 1e-12 * mass
        assert abs(sums[axis][1] - flux) <= 1e-12 * max(abs(flux), 1e-30)
    st.close()
    lat.close()


def test_a_rank_failing_between_steps_is_reported(tmp_path):
    """Rank 1 raises after its third step, with none of its kernels in
    flight; rank 0 learns of it on the host (its error or the closed
    connection ends its next exchange) and the job ends with an error."""
    with pytest.raises(Exception) as ei:
        mp.spawn(_worker, args=(2, _free_port(), str(tmp_path), "lex", 1), nprocs=2, join=True)
    msg = str(ei.value)
    assert ("failed on purpose" in msg or "Connection closed" in msg
            or "Connection reset" in msg), msg
