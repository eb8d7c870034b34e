"""Virtual ranks on one GPU: the list cut into P chunks, ghosts filled by
lbm_halo_gather from the owners' arrays before every step, each chunk
stepped on its own local adjacency (Sec. 2 and Fig. 1c: equal chunks of
the 1-D list, remote links exchanged).  The gathered result must equal the
FP64 oracle's run of the unsplit bed within the FP64 tolerance, and the
unsplit lbm_step bit for bit (same per-cell arithmetic); the per-chunk
sums must add up to the oracle's and the unsplit mass and flux."""
import numpy as np
import pytest
import torch

import fp64_measures
import oracle
from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus
from paper_1111_1129_gb300.partition import plan

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


@pytest.mark.parametrize("p", [1, 2, 3, 5, 16])
@pytest.mark.parametrize("ordering", ["lex", "blocked", "morton1"])
def test_virtual_ranks_equal_the_unsplit_run(p, ordering):
    bed = inputs.bed_small(1)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), ordering, (8, 8, 8), bed.periodic)
    n = lat.n
    adj = lat.adjacency().cpu().numpy()
    plans, send = plan(adj, n, p)
    steps, F = 9, (0.0, 0.0, 1e-5)
    ref = LBMState(lat, "f64")
    ref.step(steps, WP, WM, F)
    ref_mass, ref_flux = ref.reduce_flux(2)
    ref_f = ref.get_pdfs()
    stream = int(torch.cuda.current_stream().cuda_stream)
    w = torch.tensor([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=torch.float64, device="cuda")
    bufs, adjs, sends = [], [], []
    for pl in plans:
        a = torch.zeros(pl.local_size, dtype=torch.float64, device="cuda")
        a[:19 * pl.count] = w.repeat_interleave(pl.count)
        bufs.append([a, torch.zeros_like(a)])
        adjs.append(torch.from_numpy(pl.adj).cuda())
    for k in range(p):
        sends.append({j: torch.from_numpy(s).cuda() for j, s in send[k].items()})
    sums = torch.zeros((p, 4), dtype=torch.float64, device="cuda")
    cur = 0
    for _ in range(steps):
        for k, pl in enumerate(plans):
            for j, (off, length) in pl.recv_from.items():
                dst = bufs[k][cur].data_ptr() + 8 * (19 * pl.count + off)
                capi.lbm_halo_gather(bufs[j][cur].data_ptr(), sends[j][k].data_ptr(), length,
                                     dst, 8, stream)
        for k, pl in enumerate(plans):
            capi.lbm_step_f64_noalloc(bufs[k][cur].data_ptr(), bufs[k][cur ^ 1].data_ptr(),
                                      adjs[k].data_ptr(), pl.count, WP, WM, F, None,
                                      sums[k].data_ptr(), stream)
        cur ^= 1
    got = torch.cat([bufs[k][cur][:19 * pl.count].view(19, pl.count)
                     for k, pl in enumerate(plans)], dim=1)
    # against the oracle's dense run of the unsplit bed
    order = {"lex": oracle.ORDER_LEX, "blocked": oracle.ORDER_BLOCKED,
             "morton1": oracle.ORDER_MORTON1}[ordering]
    cells, _, adj_ref = oracle.build_sparse(bed.flags, order, (8, 8, 8), bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    np.testing.assert_array_equal(adj, adj_ref)
    f_or, obs, _, _ = oracle.run(bed.flags, bed.periodic, WP, WM, F, steps)
    m = fp64_measures.check(got.cpu().numpy(), oracle.to_sparse(f_or, cells), steps,
                            label=f"virtual ranks p={p} {ordering}")
    tot = sums.sum(dim=0).cpu().numpy()
    assert abs(tot[0] - obs[-1, 0]) <= 1e-12 * obs[-1, 0]
    assert abs(tot[3] / n - obs[-1, 3] / n) <= 11 * m["bound_abs_df"] + 2.0 ** -61
    # and the unsplit GPU run, bit for bit
    assert torch.equal(got, ref_f)
    assert abs(tot[0] - ref_mass) <= 1e-12 * ref_mass
    assert abs(tot[3] / n - ref_flux) <= 1e-12 * abs(ref_flux)
    ref.close()
    lat.close()


def test_halo_gather_element_sizes_and_validation():
    src = torch.arange(40, dtype=torch.int16, device="cuda")
    slots = torch.tensor([3, 0, 39, 7], dtype=torch.int64, device="cuda")
    dst = torch.zeros(4, dtype=torch.int16, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    capi.lbm_halo_gather(src.data_ptr(), slots.data_ptr(), 4, dst.data_ptr(), 2, stream)
    assert dst.tolist() == [3, 0, 39, 7]
    with pytest.raises(capi.LbmError):
        capi.lbm_halo_gather(src.data_ptr(), slots.data_ptr(), 4, dst.data_ptr(), 3, stream)
