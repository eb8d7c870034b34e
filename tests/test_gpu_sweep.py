"""FP64 stream-collide sweep on the GPU vs the CPU oracle (Sec. 1, 2, 7).

Tolerance: FP64 PDFs agree with the oracle to 1e-12 of max |f| (the two
sides sum in different orders; round-off is ~1e-16 per step).  Errors
relative to the deviation max |f - w| and to max |u| are printed beside it
and held to the absolute round-off bounds of fp64_measures.  Integer
outputs (step counts) and the FP64 results across orderings are compared
bit for bit.
"""
import numpy as np
import pytest
import torch

import fp64_measures
import oracle
from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


def _gpu_run(flags, periodic, steps, F, ordering="lex", block=(8, 8, 8), precision="f64",
             alpha_dense=None, f0_dense=None):
    lat = SparseLattice(torch.from_numpy(flags).cuda(), ordering, block, periodic)
    st = LBMState(lat, precision)
    cells = lat.cells().cpu().numpy()
    if f0_dense is not None:
        st.set_pdfs(torch.from_numpy(oracle.to_sparse(f0_dense, cells).copy()))
    if alpha_dense is not None:
        st.set_damping(torch.from_numpy(alpha_dense.reshape(-1)[cells].copy()))
    st.step(steps, WP, WM, F)
    return lat, st, cells


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("precision", ["f64", "f64x"])
@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 4, 5), (6, 6, 6), (5, 1, 3)])
@pytest.mark.parametrize("periodic", range(8))
def test_tiny_boxes_random_state_parity(shape, periodic, precision):
    """Brute force on tiny boxes: random flags, random initial PDFs, random
    damping, 1-10 steps, every periodicity mask; IEEE FP64 and FP64 storage
    in fixed point."""
    rng = np.random.default_rng(hash((shape, periodic)) % 2**32)
    flags = (rng.random(shape) < 0.25).astype(np.uint8)
    if (flags == 0).sum() == 0:
        flags[0, 0, 0] = 0
    f0 = oracle.rest_state(flags) * (1 + 0.05 * rng.standard_normal((19,) + shape))
    alpha = 0.05 * rng.random(shape)
    F = 1e-3 * rng.standard_normal(3)
    for steps in (1, 3, 10):
        lat, st, cells = _gpu_run(flags, periodic, steps, F, precision=precision,
                                  alpha_dense=alpha, f0_dense=f0)
        f_ref, obs, rho_ref, u_ref = oracle.run(flags, periodic, WP, WM, F, steps, alpha=alpha,
                                                f=f0)
        got = st.get_pdfs().cpu().numpy()
        rho, u = st.moments()
        fp64_measures.check(got, oracle.to_sparse(f_ref, cells), steps, u.cpu().numpy(),
                            oracle.to_sparse(u_ref, cells),
                            label=f"tiny box {shape} periodic {periodic} {precision}")
        np.testing.assert_allclose(rho.cpu().numpy(), oracle.to_sparse(rho_ref, cells),
                                   rtol=0, atol=1e-13)
        np.testing.assert_allclose(u.cpu().numpy(), oracle.to_sparse(u_ref, cells), rtol=0,
                                   atol=1e-13 * max(np.abs(u_ref).max(), 1e-30))
        mass, flux = st.reduce_flux(2)
        assert abs(mass - obs[-1, 0]) < 1e-13 * abs(obs[-1, 0])
        assert abs(flux - obs[-1, 3] / lat.n) < 1e-13 * max(np.abs(u_ref).max(), 1e-30)
        st.close()
        lat.close()


@pytest.mark.parametrize("precision", ["f64", "f64x"])
@pytest.mark.parametrize("shape", [(4, 4, 4), (4, 4, 8), (3, 43, 1), (1, 1, 65)])
def test_row_alignment_edges_parity(shape, precision):
    """Fully fluid periodic boxes of 64 and 128 cells (state rows of exactly
    N elements, read through the plain links) and of 129 and 65 cells (rows
    padded to 192 and 128 elements, read through the padded links): random
    state, damping and force against the oracle."""
    rng = np.random.default_rng(sum(shape))
    flags = np.zeros(shape, np.uint8)
    f0 = oracle.rest_state(flags) * (1 + 0.05 * rng.standard_normal((19,) + shape))
    alpha = 0.05 * rng.random(shape)
    F = 1e-3 * rng.standard_normal(3)
    for steps in (1, 4):
        lat, st, cells = _gpu_run(flags, 7, steps, F, precision=precision, alpha_dense=alpha,
                                  f0_dense=f0)
        assert lat.n == flags.size
        f_ref, obs, _, u_ref = oracle.run(flags, 7, WP, WM, F, steps, alpha=alpha, f=f0)
        rho, u = st.moments()
        fp64_measures.check(st.get_pdfs().cpu().numpy(), oracle.to_sparse(f_ref, cells), steps,
                            u.cpu().numpy(), oracle.to_sparse(u_ref, cells),
                            label=f"box {shape} {precision}")
        mass, flux = st.reduce_flux(0)
        assert abs(mass - obs[-1, 0]) < 1e-13 * abs(obs[-1, 0])
        assert abs(flux - obs[-1, 1] / lat.n) < 1e-13 * max(np.abs(u_ref).max(), 1e-30)
        st.close()
        lat.close()


@pytest.mark.parametrize("precision", ["f64", "f32s"])
def test_reduction_of_large_moments_takes_the_fp64_path(precision):
    """States far from rest (|rho - 1| and |u| up to ~1): warps holding a
    value >= 1/4 sum in FP64 instead of fixed point, mixed with warps that
    do not; mass and flux must still match the oracle."""
    rng = np.random.default_rng(11)
    shape = (12, 10, 9)
    flags = (rng.random(shape) < 0.2).astype(np.uint8)
    f0 = oracle.rest_state(flags) * (1 + 0.02 * rng.standard_normal((19,) + shape))
    hot = rng.random(shape) < 0.1           # a tenth of the cells far from rest
    f0[:, hot] *= 1 + 0.9 * rng.random((19, int(hot.sum())))
    F = (1e-3, -2e-3, 3e-3)
    lat, st, cells = _gpu_run(flags, 0b111, 1, F, precision=precision, f0_dense=f0)
    _, obs, rho_ref, u_ref = oracle.run(flags, 0b111, WP, WM, F, 1, f=f0)
    rho_s = oracle.to_sparse(rho_ref, cells)
    assert np.abs(rho_s - 1).max() >= 0.25     # the FP64 path is taken
    tol = 1e-13 if precision == "f64" else 1e-6
    mass, _ = st.reduce_flux(0)
    assert abs(mass - obs[-1, 0]) <= tol * abs(obs[-1, 0])
    for axis in range(3):
        _, flux = st.reduce_flux(axis)
        ref = obs[-1, 1 + axis] / lat.n
        assert abs(flux - ref) <= tol * np.abs(u_ref).max(), (axis, flux, ref)
    st.close()
    lat.close()


def test_small_bed_1000_steps_parity():
    """The 32x32x64 packed bed, lexicographic order, 1000 FP64 steps from
    rest with F = 1e-6 along z."""
    bed = inputs.bed_small(0)
    F = (0.0, 0.0, 1e-6)
    steps = 1000
    lat, st, cells = _gpu_run(bed.flags, bed.periodic, steps, F)
    f_ref, obs, rho_ref, u_ref = oracle.run(bed.flags, bed.periodic, WP, WM, F, steps)
    got = st.get_pdfs().cpu().numpy()
    rho, u = st.moments()
    m = fp64_measures.check(got, oracle.to_sparse(f_ref, cells), steps, u.cpu().numpy(),
                            oracle.to_sparse(u_ref, cells), label="small bed, 1000 steps")
    mass, flux = st.reduce_flux(2)
    assert abs(mass - obs[-1, 0]) < 1e-12 * obs[-1, 0]
    assert abs(flux - obs[-1, 3] / bed.n_fluid) <= m["bound_abs_du"] + 2.0 ** -61
    assert st.steps == steps
    st.close()
    lat.close()


def test_orderings_give_bitwise_identical_fields():
    """The per-cell arithmetic does not depend on the cell order, so every
    numbering scheme yields the same FP64 field, bit for bit."""
    bed = inputs.bed_small(2)
    F = (0.0, 0.0, 1e-5)
    ref = None
    for ordering, block in [("lex", (1, 1, 1)), ("blocked", (8, 8, 8)), ("blocked", (4, 2, 16)),
                            ("morton1", (1, 1, 1)), ("morton2", (1, 1, 1))]:
        lat, st, cells = _gpu_run(bed.flags, bed.periodic, 100, F, ordering, block)
        dense = np.zeros((19, bed.flags.size))
        dense[:, cells] = st.get_pdfs().cpu().numpy()
        if ref is None:
            ref = dense
        else:
            np.testing.assert_array_equal(dense, ref)
        st.close()
        lat.close()


@pytest.mark.parametrize("precision", ["f64", "f64x"])
def test_damped_bed_parity(precision):
    bed = inputs.packed_bed((24, 20, 28), 2, 18.0, 3.0, 0.45, 5)
    alpha = inputs.alpha_field(bed.dims, seed=5)
    F = (0.0, 0.0, 1e-5)
    lat, st, cells = _gpu_run(bed.flags, bed.periodic, 200, F, "morton1", precision=precision,
                              alpha_dense=alpha)
    f_ref, obs, _, u_ref = oracle.run(bed.flags, bed.periodic, WP, WM, F, 200, alpha=alpha)
    _, u = st.moments()
    m = fp64_measures.check(st.get_pdfs().cpu().numpy(), oracle.to_sparse(f_ref, cells), 200,
                            u.cpu().numpy(), oracle.to_sparse(u_ref, cells),
                            label=f"damped bed, 200 steps, {precision}")
    mass, flux = st.reduce_flux(2)
    assert abs(flux - obs[-1, 3] / bed.n_fluid) <= m["bound_abs_du"] + 2.0 ** -61
    st.close()
    lat.close()


def test_reductions_are_deterministic_and_need_a_step():
    bed = inputs.bed_small(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "blocked", (8, 8, 8), bed.periodic)
    vals = []
    for _ in range(2):
        st = LBMState(lat, "f64")
        with pytest.raises(capi.LbmError):
            st.reduce_flux(2)
        st.step(50, WP, WM, (0, 0, 1e-6))
        vals.append(st.reduce_flux(2))
        with pytest.raises(capi.LbmError):
            st.reduce_flux(3)
        st.close()
    assert vals[0] == vals[1]
    lat.close()


def test_state_roundtrip_and_rest_init():
    bed = inputs.bed_small(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    st = LBMState(lat, "f64")
    _, w, _ = oracle.velocity_set()
    f = st.get_pdfs().cpu().numpy()
    np.testing.assert_array_equal(f, np.repeat(w[:, None], lat.n, axis=1))
    rng = np.random.default_rng(0)
    f1 = rng.random((19, lat.n))
    st.set_pdfs(torch.from_numpy(f1))
    np.testing.assert_array_equal(st.get_pdfs().cpu().numpy(), f1)
    assert st.steps == 0
    st.close()
    lat.close()


def test_empty_domain_steps():
    flags = np.ones((3, 4, 5), np.uint8)
    lat = SparseLattice(torch.from_numpy(flags).cuda(), "lex")
    st = LBMState(lat, "f64")
    st.step(3, WP, WM, (0, 0, 1e-6))
    assert st.reduce_flux(0) == (0.0, 0.0)
    st.close()
    lat.close()


def test_step_argument_validation():
    bed = inputs.bed_small(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    st = LBMState(lat, "f64")
    for bad in [dict(n_steps=-1), dict(omega_plus=2.0), dict(omega_minus=0.0),
                dict(force=(0.0, float("nan"), 0.0))]:
        args = dict(n_steps=1, omega_plus=WP, omega_minus=WM, force=(0, 0, 1e-6))
        args.update(bad)
        with pytest.raises(capi.LbmError) as ei:
            st.step(**args)
        assert ei.value.status == capi.LBM_EINVAL
    st.close()
    lat.close()


@pytest.mark.parametrize("ordering", ["lex", "blocked"])
def test_large_bed_sampled_parity(ordering):
    """The 1024x256x256 bed at full size, in lexicographic order (the launch
    configuration the benchmark times) and 8^3 blocked order: adjacency
    bit-exact against the oracle, and one step checked cell by cell on a
    sample with the oracle's collision applied to the oracle's own pull of
    the GPU's previous state."""
    bed = inputs.bed_large(0)
    kind = {"lex": oracle.ORDER_LEX, "blocked": oracle.ORDER_BLOCKED}[ordering]
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), ordering, (8, 8, 8), bed.periodic)
    cells, _, adj = oracle.build_sparse(bed.flags, kind, (8, 8, 8), bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    np.testing.assert_array_equal(lat.adjacency().cpu().numpy(), adj)
    st = LBMState(lat, "f64")
    F = (1e-6, 0.0, 0.0)
    st.step(20, WP, WM, F)
    prev = st.get_pdfs().cpu().numpy().ravel()
    st.step(1, WP, WM, F)
    nxt = st.get_pdfs().cpu().numpy()
    mass, _ = st.reduce_flux(0)
    assert abs(mass - lat.n) < 1e-10 * lat.n
    rng = np.random.default_rng(0)
    sample = rng.choice(lat.n, 2000, replace=False)
    ref = np.empty((19, sample.size))
    for j, n in enumerate(sample):
        g = np.concatenate([[prev[n]], prev[adj[:, n]]])
        ref[:, j], _, _ = oracle.collide(g, F, 0.0, WP, WM)
    fp64_measures.check(nxt[:, sample], ref, 1, label=f"large bed {ordering}, one step, 2000 cells")
    st.close()
    lat.close()
