"""GPU assembly of the sparse representation vs the CPU oracle: numbering
keys, contiguous index and adjacency must match bit for bit (Sec. 2-3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1111_1129_gb300 import SparseLattice, build, capi, inputs, ordering_keys

pytestmark = pytest.mark.gpu

ORDERS = [("lex", (1, 1, 1), oracle.ORDER_LEX),
          ("blocked", (8, 8, 8), oracle.ORDER_BLOCKED),
          ("blocked", (2, 3, 5), oracle.ORDER_BLOCKED),
          ("blocked", (64, 64, 64), oracle.ORDER_BLOCKED),
          ("morton1", (1, 1, 1), oracle.ORDER_MORTON1),
          ("morton2", (1, 1, 1), oracle.ORDER_MORTON2),
          ("hilbert", (1, 1, 1), oracle.ORDER_HILBERT)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()
    torch.cuda.init()


def _random_flags(shape, solid, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(shape) < solid).astype(np.uint8)


def _check_against_oracle(flags, name, block, kind, periodic):
    lat = SparseLattice(torch.from_numpy(flags).cuda(), name, block, periodic)
    cells, inv, adj = oracle.build_sparse(flags, kind, block, periodic)
    assert lat.n == len(cells)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    np.testing.assert_array_equal(lat.inverse().cpu().numpy(), inv)
    np.testing.assert_array_equal(lat.adjacency().cpu().numpy(), adj)
    lat.close()


@pytest.mark.parametrize("name,block,kind", ORDERS)
@pytest.mark.parametrize("dims", [(37, 29, 23), (64, 16, 8), (1, 1, 1), (5, 1, 200)])
def test_keys_bit_exact(name, block, kind, dims):
    got = ordering_keys(dims, name, block).cpu().numpy().astype(np.uint64)
    np.testing.assert_array_equal(got, oracle.keys(kind, dims, block))


@pytest.mark.parametrize("name,block,kind", ORDERS)
@pytest.mark.parametrize("periodic", [0, 1, 2, 4, 7])
def test_sparse_bit_exact_random_flags(name, block, kind, periodic):
    # 37x29x23 = 24679 cells: several 4096-key tiles plus a ragged tail
    flags = _random_flags((23, 29, 37), 0.35, 100 + periodic + 7 * kind)
    _check_against_oracle(flags, name, block, kind, periodic)


@pytest.mark.parametrize("name,block,kind", [ORDERS[0], ORDERS[1], ORDERS[4], ORDERS[5]])
def test_sparse_bit_exact_packed_beds(name, block, kind):
    for bed in (inputs.bed_small(0), inputs.bed_medium(0)):
        _check_against_oracle(bed.flags, name, block, kind, bed.periodic)


@pytest.mark.parametrize("shape", [(23, 29, 37), (2, 3, 4096), (1, 1, 17)])
def test_lex_vector_and_generic_passes_agree(shape):
    """Lexicographic order with 16-byte aligned flags takes the vector passes
    (16 flags per thread); flags at an odd address take the generic key
    walk.  Both give the oracle's representation, through full chunks,
    whole 4096-key tiles and a ragged tail."""
    flags = _random_flags(shape, 0.3, sum(shape))
    cells, inv, adj = oracle.build_sparse(flags, oracle.ORDER_LEX, (1, 1, 1), 5)
    buf = torch.zeros(flags.size + 16, dtype=torch.uint8, device="cuda")
    for off in (0, 1):
        view = buf[off:off + flags.size]
        view.copy_(torch.from_numpy(flags.reshape(-1)).cuda())
        assert (view.data_ptr() % 16 == 0) == (off == 0)
        lat = SparseLattice(view.reshape(shape), "lex", periodic=5)
        np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
        np.testing.assert_array_equal(lat.inverse().cpu().numpy(), inv)
        np.testing.assert_array_equal(lat.adjacency().cpu().numpy(), adj)
        lat.close()


def test_cells_follow_key_order():
    bed = inputs.bed_small(1)
    for name, block, kind in ORDERS:
        lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), name, block, bed.periodic)
        keys = ordering_keys(bed.dims, name, block).reshape(-1)
        k = keys[lat.cells().long()].cpu().numpy().astype(np.uint64)
        assert np.all(k[1:] > k[:-1])
        lat.close()


def test_degenerate_domains():
    solid = np.ones((4, 5, 6), np.uint8)
    lat = SparseLattice(torch.from_numpy(solid).cuda(), "morton1")
    assert lat.n == 0
    assert np.all(lat.inverse().cpu().numpy() == -1)
    lat.close()
    one = np.zeros((1, 1, 1), np.uint8)
    lat = SparseLattice(torch.from_numpy(one).cuda(), "lex", periodic=7)
    np.testing.assert_array_equal(lat.adjacency().cpu().numpy()[:, 0], np.arange(1, 19))
    lat.close()
    lat = SparseLattice(torch.from_numpy(one).cuda(), "lex", periodic=0)
    opp = oracle.velocity_set()[2]
    np.testing.assert_array_equal(lat.adjacency().cpu().numpy()[:, 0], opp[1:])
    lat.close()


def test_bad_flags_are_rejected():
    flags = np.zeros((4, 4, 4), np.uint8)
    flags[1, 2, 3] = 2
    with pytest.raises(capi.LbmError) as ei:
        SparseLattice(torch.from_numpy(flags).cuda(), "lex")
    assert ei.value.status == capi.LBM_EFLAGS


def test_ordering_tuner_on_a_sample():
    from paper_1111_1129_gb300.autotune import DEFAULT_CANDIDATES, tune_ordering
    bed = inputs.bed_medium(0)
    best, table = tune_ordering(bed.flags, 0, bed.periodic, sample_length=32, steps=5)
    assert len(table) == len(DEFAULT_CANDIDATES)
    assert best == table[0][:2] and best in [(n, tuple(b)) for n, b in DEFAULT_CANDIDATES]
    assert all(r[2] > 0 for r in table)
    assert [r[2] for r in table] == sorted((r[2] for r in table), reverse=True)


@pytest.mark.parametrize("pinned", [False, True])
def test_build_from_host_flags(pinned):
    """lbm_build_sparse takes host flags (pageable or pinned) as well as
    device flags; the result is the same representation bit for bit."""
    from paper_1111_1129_gb300.lbm import ORDERINGS, _borrow
    bed = inputs.packed_bed((40, 36, 30), 2, 28.0, 4.0, 0.45, 6)
    flags = torch.from_numpy(bed.flags)
    if pinned:
        flags = flags.pin_memory()
    stream = int(torch.cuda.current_stream().cuda_stream)
    h = capi.lbm_build_sparse(flags.data_ptr(), bed.dims,
                              capi.make_ordering(ORDERINGS["morton1"], (1, 1, 1), bed.periodic),
                              stream)
    n, cells_p, adj_p, inv_p = capi.lbm_sparse_info(h)
    cells, inv, adj = oracle.build_sparse(bed.flags, oracle.ORDER_MORTON1, (1, 1, 1),
                                          bed.periodic)
    assert n == len(cells)
    np.testing.assert_array_equal(_borrow(cells_p, (n,), "<i4", torch.int32).cpu().numpy(), cells)
    np.testing.assert_array_equal(_borrow(adj_p, (18, n), "<i4", torch.int32).cpu().numpy(), adj)
    np.testing.assert_array_equal(
        _borrow(inv_p, bed.flags.shape, "<i4", torch.int32).cpu().numpy(), inv)
    capi.lbm_free(h)
