"""The fixed-point FP64-storage sweep (LBM_F64X) against the oracle and the
IEEE FP64 path.  It must agree with the oracle within the FP64 tolerance
(1e-12 of max |f|), conserve the stored mass exactly (the sum over all
slots of bits(f_q) - bits(w_q), in units of 2^-58, never changes), and give
the same field under every cell ordering."""
import numpy as np
import pytest
import torch

import fp64_measures
import oracle
from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
WBITS = np.array([0x3FD5555555555555] + [0x3FAC71C71C71C71C] * 6 + [0x3F9C71C71C71C71C] * 12,
                 dtype=np.int64)
SHIFT = np.array([4] + [1] * 6 + [0] * 12, dtype=np.int64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


def _units(f):
    """Exact stored deviations in units of 2^-58 (all values in range)."""
    bits = np.ascontiguousarray(f).view(np.int64)
    assert np.all((bits >> 52) == (WBITS[:, None] >> 52))
    return (bits - WBITS[:, None]) << SHIFT[:, None]


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_small_bed_parity_and_exact_mass():
    bed = inputs.bed_small(0)
    F = (0.0, 0.0, 1e-6)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    cells = lat.cells().cpu().numpy()
    st = LBMState(lat, "f64x")
    st64 = LBMState(lat, "f64")
    totals = []
    for _ in range(10):
        st.step(100, WP, WM, F)
        st64.step(100, WP, WM, F)
        totals.append(sum(_units(st.get_pdfs().cpu().numpy()).ravel().tolist()))
    assert totals == [0] * 10                       # exact mass conservation
    f_ref, obs, _, u_ref = oracle.run(bed.flags, bed.periodic, WP, WM, F, 1000)
    got = st.get_pdfs().cpu().numpy()
    _, u = st.moments()
    m = fp64_measures.check(got, oracle.to_sparse(f_ref, cells), 1000, u.cpu().numpy(),
                            oracle.to_sparse(u_ref, cells), label="f64x small bed, 1000 steps")
    assert _rel(got, st64.get_pdfs().cpu().numpy()) < 1e-13
    mass, flux = st.reduce_flux(2)
    assert abs(flux - obs[-1, 3] / bed.n_fluid) <= m["bound_abs_du"] + 2.0 ** -61
    assert abs(mass - bed.n_fluid) < 1e-12 * bed.n_fluid
    st.close()
    st64.close()
    lat.close()


@pytest.mark.parametrize("shape,periodic", [((3, 4, 5), 0b100), ((6, 6, 6), 0b111),
                                            ((5, 1, 3), 0b000)])
def test_out_of_range_cells_fall_back_to_fp64(shape, periodic):
    """Random states with 20% perturbations put many PDFs outside their
    binary range; those cells take the IEEE path."""
    rng = np.random.default_rng(sum(shape))
    flags = (rng.random(shape) < 0.25).astype(np.uint8)
    f0 = oracle.rest_state(flags) * (1 + 0.2 * rng.standard_normal((19,) + shape))
    F = 1e-3 * rng.standard_normal(3)
    lat = SparseLattice(torch.from_numpy(flags).cuda(), "morton1", periodic=periodic)
    cells = lat.cells().cpu().numpy()
    st = LBMState(lat, "f64x")
    st.set_pdfs(torch.from_numpy(oracle.to_sparse(f0, cells).copy()))
    st.step(5, WP, WM, F)
    f_ref, obs, _, _ = oracle.run(flags, periodic, WP, WM, F, 5, f=f0)
    # values up to ~0.6 here (ulp 2^-53): the relative measure is the bound
    m = fp64_measures.measures(st.get_pdfs().cpu().numpy(), oracle.to_sparse(f_ref, cells), 5,
                               label=f"f64x fallback {shape}")
    assert m["rel_to_max_f"] < 1e-12, m
    # the reduction adds the IEEE-path cells' FP64 moments to the warp slots
    # that the fixed-point cells wrote
    n = lat.n
    for axis in range(3):
        mass, flux = st.reduce_flux(axis)
        assert abs(mass - obs[-1, 0]) <= 1e-12 * abs(obs[-1, 0])
        assert abs(flux - obs[-1, 1 + axis] / n) <= 1e-12 * max(1.0, abs(obs[-1, 1:]).max() / n)
    st.close()
    lat.close()


def test_orderings_bitwise_identical():
    bed = inputs.bed_small(2)
    ref = None
    for ordering, block in [("lex", (1, 1, 1)), ("blocked", (8, 8, 8)), ("morton2", (1, 1, 1))]:
        lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), ordering, block, bed.periodic)
        st = LBMState(lat, "f64x")
        st.step(200, WP, WM, (0.0, 0.0, 1e-5))
        dense = np.zeros((19, bed.flags.size))
        dense[:, lat.cells().cpu().numpy()] = st.get_pdfs().cpu().numpy()
        if ref is None:
            ref = dense
        else:
            np.testing.assert_array_equal(dense, ref)
        st.close()
        lat.close()


@pytest.mark.parametrize("ordering", ["lex", "blocked"])
def test_large_bed_sampled_parity(ordering):
    """1024x256x256 bed in lexicographic order (the benchmark's launch
    configuration) and 8^3 blocked order: one step checked cell by cell
    with the oracle's collision on a sample, and the stored mass unchanged
    exactly after 50 steps."""
    bed = inputs.bed_large(0)
    kind = {"lex": oracle.ORDER_LEX, "blocked": oracle.ORDER_BLOCKED}[ordering]
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), ordering, (8, 8, 8), bed.periodic)
    cells, _, adj = oracle.build_sparse(bed.flags, kind, (8, 8, 8), bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    st = LBMState(lat, "f64x")
    F = (1e-6, 0.0, 0.0)
    st.step(49, WP, WM, F)
    prev = st.get_pdfs().cpu().numpy()
    st.step(1, WP, WM, F)
    nxt = st.get_pdfs().cpu().numpy()
    assert int(_units(nxt).sum(dtype=np.int64)) == 0
    flat = prev.ravel()
    rng = np.random.default_rng(1)
    sample = rng.choice(lat.n, 2000, replace=False)
    ref = np.empty((19, sample.size))
    for j, n in enumerate(sample):
        g = np.concatenate([[flat[n]], flat[adj[:, n]]])
        ref[:, j], _, _ = oracle.collide(g, F, 0.0, WP, WM)
    # a few ulp of the rest population (~0.33, ulp 5.6e-17): it takes the
    # rounding of rho and the oracle rounds too
    fp64_measures.check(nxt[:, sample], ref, 1, label=f"f64x large bed {ordering}, one step, 2000 cells")
    st.close()
    lat.close()


def test_strong_damping_takes_the_ieee_path_where_needed():
    """Damping drawn in [0, 1] on a random-flag box near rest: cells with
    alpha >= 1/2 take the IEEE collision, the others the fixed-point one;
    both match the oracle within the FP64 tolerance."""
    rng = np.random.default_rng(31)
    shape = (10, 9, 12)
    flags = (rng.random(shape) < 0.2).astype(np.uint8)
    alpha = rng.random(shape)
    f0 = oracle.rest_state(flags) * (1 + 1e-4 * rng.standard_normal((19,) + shape))
    F = (1e-5, -2e-5, 3e-5)
    lat = SparseLattice(torch.from_numpy(flags).cuda(), "lex", periodic=0b110)
    cells = lat.cells().cpu().numpy()
    st = LBMState(lat, "f64x")
    st.set_pdfs(torch.from_numpy(oracle.to_sparse(f0, cells).copy()))
    st.set_damping(torch.from_numpy(alpha.reshape(-1)[cells].copy()))
    st.step(15, WP, WM, F)
    f_ref, obs, _, u_ref = oracle.run(flags, 0b110, WP, WM, F, 15, alpha=alpha, f=f0)
    _, u = st.moments()
    fp64_measures.check(st.get_pdfs().cpu().numpy(), oracle.to_sparse(f_ref, cells), 15,
                        u.cpu().numpy(), oracle.to_sparse(u_ref, cells),
                        label="f64x strong damping")
    st.close()
    lat.close()
