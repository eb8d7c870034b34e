"""Batched beds against the FP64 oracle, bed by bed.

Many packed beds of uneven sizes are concatenated into one list and stepped
by one launch per step, each bed with its own body force, on the sparse
representation with implicit bounce back (Sec. 2).  The beds: cube sides
drawn in 12..33, sphere radii in 2.5..5, a tube along z, and one bed with
no fluid at all, 8^3-blocked order.  Every bed is compared with the oracle
run on that bed alone:

* FP64 storage, 25 steps from rest: PDFs within the FP64 tolerance (1e-12
  of max |f|, plus the absolute round-off bounds of fp64_measures), mass
  within 1e-12 and the mean velocity along each axis within the velocity
  round-off bound, with all beds in one launch group and in L2-sized
  groups, at two launch shapes, with and without graph replay;
* FP32 / FP16 / BF16 shifted storage: one step from a random
  non-equilibrium state read back from the form, every output within one
  storage unit (plus the FP32 rounding of the collision) of the oracle's
  sparse stepper on the bed's own adjacency.
"""
import numpy as np
import pytest
import torch

import fp64_measures
import oracle
from paper_1111_1129_gb300 import (BatchedState, SparseLattice, build, capi, inputs,
                                   omega_minus, shifted_scale_exp)
from storage_units import W, codes_equal_fraction, one_step_tolerance

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
BLOCK = (8, 8, 8)


@pytest.fixture(scope="module")
def batch():
    build.build()
    capi.load()
    rng = np.random.default_rng(2)
    beds = []
    for b in range(7):
        s = int(rng.integers(12, 34))
        beds.append(inputs.packed_bed((s, s, s), 2, s - 2.0, float(rng.uniform(2.5, 5)), 0.0,
                                      100 + b))
    beds.insert(3, inputs.packed_bed((8, 8, 8), 2, 0.5, 0.0, 0.0, 0))   # no fluid
    forces = [(1e-6 * (b + 1), -2e-7 * b, 1e-5 / (b + 1)) for b in range(len(beds))]
    lats, ref = [], []
    for bed in beds:
        lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "blocked", BLOCK, bed.periodic)
        cells, _, adj = oracle.build_sparse(bed.flags, oracle.ORDER_BLOCKED, BLOCK, bed.periodic)
        np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
        lats.append(lat)
        ref.append((cells, adj))
    assert lats[3].n == 0
    yield beds, forces, lats, ref
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("block,cpt,graph,group_bytes", [(256, 2, True, 0), (512, 4, False, -1),
                                                         (128, 1, True, 1)])
def test_fp64_batch_matches_the_oracle_bed_by_bed(batch, block, cpt, graph, group_bytes):
    beds, forces, lats, ref = batch
    steps = 25
    bs = BatchedState(lats, "f64")
    bs.configure(block, cpt, graph)
    bs.groups(group_bytes)
    bs.step(steps, WP, WM, forces)
    sums = [bs.reduce_flux(axis) for axis in range(3)]
    f_all = bs.get_pdfs().cpu().numpy()
    for i, (bed, F, (cells, _)) in enumerate(zip(beds, forces, ref)):
        b, c = bs.begin[i], bs.count[i]
        assert c == cells.size
        if c == 0:
            assert all(s[0][i] == 0.0 and s[1][i] == 0.0 for s in sums)
            continue
        f_ref, obs, _, u_ref = oracle.run(bed.flags, bed.periodic, WP, WM, F, steps)
        m = fp64_measures.check(f_all[:, b:b + c], oracle.to_sparse(f_ref, cells), steps,
                                label=f"batched bed {i} (N={c}), {block}x{cpt}, "
                                      f"groups {group_bytes}")
        mass = sums[0][0][i]
        assert abs(mass - obs[-1, 0]) <= 1e-12 * obs[-1, 0], (i, mass, obs[-1, 0])
        for axis in range(3):
            flux_ref = obs[-1, 1 + axis] / c
            # the mean of per-cell velocities is off by at most the largest
            # per-cell velocity error, plus the fixed-point unit 2^-61
            bound = 11 * m["bound_abs_df"] + 2.0 ** -61
            assert abs(sums[axis][1][i] - flux_ref) <= bound, (i, axis, sums[axis][1][i],
                                                               flux_ref)
    bs.close()


@pytest.mark.parametrize("precision", ["f32s", "f16s", "bf16s"])
def test_reduced_forms_one_step_within_one_storage_unit(batch, precision):
    beds, forces, lats, ref = batch
    dev = 1e-4
    k = shifted_scale_exp(4 * dev)
    assert k <= 33   # keeps w + code * 2^-k exact in FP64
    bs = BatchedState(lats, precision, k)
    rng = np.random.default_rng(17)
    f0 = np.repeat(W[:, None], bs.n_padded, axis=1)
    for b, c in zip(bs.begin, bs.count):
        f0[:, b:b + c] += dev * rng.uniform(-1.0, 1.0, size=(19, c))
    f0_dev = torch.from_numpy(f0).cuda().contiguous()
    capi.lbm_state_set_pdfs(bs.handle, f0_dev.data_ptr())
    f_rep = bs.get_pdfs().cpu().numpy()       # what the form stores, decoded exactly
    bs.step(1, WP, WM, forces)
    f_gpu = bs.get_pdfs().cpu().numpy()
    bs.close()
    for i, (F, (cells, adj)) in enumerate(zip(forces, ref)):
        b, c = bs.begin[i], bs.count[i]
        if c == 0:
            continue
        rep = np.ascontiguousarray(f_rep[:, b:b + c])
        got = f_gpu[:, b:b + c]
        f_ref = oracle.sparse_step(rep, adj, c, F, WP, WM).reshape(19, c)
        tol = one_step_tolerance(precision, f_ref, float(np.abs(rep - W[:, None]).max()), k)
        worst = float((np.abs(got - f_ref) / tol).max())
        print(f"{precision} bed {i} N={c}: max err/tol {worst:.3f}")
        assert np.isfinite(got).all()
        assert worst <= 1.0, (precision, i, worst)
        if precision != "f32s":
            same = codes_equal_fraction(precision, got, f_ref, k)
            assert same >= 0.99, (precision, i, same)
