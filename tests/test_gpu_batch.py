"""Batched beds (one launch per step over concatenated cell lists, per-bed
forces, CUDA graph, tuned launch shape, L2 groups of beds stepped one group
at a time, resident steps that keep the links in shared memory across a
call's steps): every bed's PDFs and flux must be bit-identical to stepping
that bed alone, whatever the launch shape, the grouping and the mode."""
import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import (BatchedState, LBMState, SparseLattice, build, capi, inputs,
                                   omega_minus)

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


def _beds(n=7, seed=2):
    rng = np.random.default_rng(seed)
    beds = []
    for b in range(n):
        s = int(rng.integers(12, 34))
        beds.append(inputs.packed_bed((s, s, s), 2, s - 2.0, float(rng.uniform(2.5, 5)), 0.0,
                                      100 + b))
    # one bed with no fluid at all
    beds.append(inputs.packed_bed((8, 8, 8), 2, 0.5, 0.0, 0.0, 0))
    forces = [(1e-6 * (b + 1), -2e-7 * b, 1e-5 / (b + 1)) for b in range(len(beds))]
    return beds, forces


def _lattices(beds):
    return [SparseLattice(torch.from_numpy(b.flags).cuda(), "blocked", (8, 8, 8), b.periodic)
            for b in beds]


@pytest.mark.parametrize("precision", ["f64", "f32s", "f16s", "bf16s"])
def test_batched_beds_bit_identical_to_separate_runs(precision):
    beds, forces = _beds()
    lats = _lattices(beds)
    assert lats[-1].n == 0
    steps = 37
    ref_f, ref_flux = [], []
    for lat, F in zip(lats, forces):
        st = LBMState(lat, precision, 20)
        st.step(steps, WP, WM, F)
        ref_f.append(st.get_pdfs().cpu().numpy())
        ref_flux.append(st.reduce_flux(2) if lat.n > 0 else None)
        st.close()
    for block, cpt, graph, group_bytes in [(256, 1, True, 0), (128, 4, True, 0),
                                           (512, 2, False, 0), (512, 4, True, 0),
                                           (256, 1, True, 1), (256, 2, True, 3 << 20),
                                           (128, 2, True, 1), (512, 4, False, 1 << 20)]:
        bs = BatchedState(lats, precision, 20)
        bs.configure(block, cpt, graph)
        n_groups = bs.groups(group_bytes)
        if group_bytes == 0:
            assert n_groups == 1
        if group_bytes == 1:
            assert n_groups == sum(1 for lat in lats if lat.n > 0)
        bs.step(steps, WP, WM, forces)
        mass, flux = bs.reduce_flux(2)
        f_all = bs.get_pdfs().cpu().numpy()
        for i in range(len(lats)):
            b, c = bs.begin[i], bs.count[i]
            assert b % 2048 == 0
            np.testing.assert_array_equal(f_all[:, b:b + c], ref_f[i])
            if ref_flux[i] is not None:
                assert (mass[i], flux[i]) == ref_flux[i]
            else:
                assert (mass[i], flux[i]) == (0.0, 0.0)
        bs.close()
    for lat in lats:
        lat.close()


def test_group_split_follows_the_budget():
    """Groups are runs of consecutive beds whose padded cells times the bytes
    per cell (two PDF grids and 18 int32 links) fit the budget; a bed above
    it is alone; an empty bed joins no group."""
    beds, _ = _beds(7, seed=5)
    lats = _lattices(beds)
    for precision, per_cell in (("f32s", 2 * 19 * 4 + 72), ("f16s", 2 * 19 * 2 + 72),
                                ("f64", 2 * 19 * 8 + 72)):
        bs = BatchedState(lats, precision, 20)
        spans = [(c + 2047) // 2048 * 2048 for c in bs.count]
        for budget in (1, 2048 * per_cell, 3 * 2048 * per_cell, 10 * 2048 * per_cell, 0):
            expect, cur = 0, 0
            for s_ in spans:
                if s_ == 0:
                    continue
                if cur > 0 and (cur + s_) * per_cell > budget:
                    expect += 1
                    cur = 0
                cur += s_
            expect += 1
            if budget == 0:
                expect = 1
            assert bs.groups(budget) == expect, (precision, budget)
        assert bs.groups(-1) >= 1
        bs.close()
    for lat in lats:
        lat.close()


def test_graph_replay_follows_new_forces():
    beds, forces = _beds(4, seed=3)
    lats = _lattices(beds)
    bs = BatchedState(lats, "f32s")
    bs.step(10, WP, WM, forces)
    forces2 = [(f[0] * 3, f[1], -f[2]) for f in forces]
    bs.step(10, WP, WM, forces2)          # same K: the cached graph is replayed
    _, flux = bs.reduce_flux(2)
    for i, lat in enumerate(lats[:-1]):
        st = LBMState(lat, "f32s")
        st.step(10, WP, WM, forces[i])
        st.step(10, WP, WM, forces2[i])
        assert st.reduce_flux(2)[1] == flux[i]
        st.close()
    bs.close()
    for lat in lats:
        lat.close()


def test_tuner_picks_a_candidate_and_keeps_results():
    beds, forces = _beds(5, seed=4)
    lats = _lattices(beds)
    a = BatchedState(lats, "f32s")
    block, cpt, ms = a.tune(3, WP, WM, forces)
    assert block in (128, 256, 512) and cpt in (1, 2, 4)
    assert len(ms) == 9 and min(ms) > 0
    taken = 9 * 4
    b = BatchedState(lats, "f32s")
    b.configure(256, 1, False)
    b.step(taken, WP, WM, forces)
    np.testing.assert_array_equal(a.get_pdfs().cpu().numpy(), b.get_pdfs().cpu().numpy())
    a.close()
    b.close()
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("group_bytes,resident,precision",
                         [(0, 0, "f32s"), (-1, 0, "f32s"), (-1, 1, "f32s"), (-1, 1, "f16s")])
def test_full_batch_of_256_beds_sampled(group_bytes, resident, precision):
    """The 256-bed workload (cube sides uniform in {24..96}, radii in [3, 8],
    forces in [1e-7, 1e-5] along z), 1000 steps, as one graph (one group), in
    the default L2 groups, and with resident steps in groups of up to the
    resident capacity (runs of ~3,200 cells that cross bed boundaries):
    per-bed flux of 8 sampled beds equals their separate runs."""
    beds, fz = inputs.batch_beds(256, 0)
    forces = [(0.0, 0.0, float(f)) for f in fz]
    lats = _lattices(beds)
    k = 19 if precision == "f16s" else 0
    bs = BatchedState(lats, precision, k)
    bs.configure(256, 2, True)
    n_groups = bs.groups(group_bytes)
    assert (n_groups == 1) == (group_bytes == 0)
    if resident:
        n_groups, cap = bs.resident(1)
        assert n_groups > 1 and cap >= 100_000
        assert n_groups * cap >= bs.n_padded
    bs.step(1000, WP, WM, forces)
    mass, flux = bs.reduce_flux(2)
    assert bs.n_fluid == sum(b.n_fluid for b in beds)
    rng = np.random.default_rng(group_bytes + 1 + resident)
    for i in rng.choice(256, 8, replace=False):
        st = LBMState(lats[i], precision, k)
        st.step(1000, WP, WM, forces[i])
        assert st.reduce_flux(2) == (mass[i], flux[i])
        st.close()
    bs.close()
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("precision", ["f32", "f32s", "f16s", "bf16s"])
def test_resident_steps_bit_identical_to_separate_runs(precision):
    """Resident steps under several groupings and call lengths (1, 2, 3 and
    37 steps; the mode switched off and on between calls) give every bed the
    PDFs and flux of its separate run."""
    beds, forces = _beds()
    lats = _lattices(beds)
    calls = [37, 1, 2, 3]
    ref_f, ref_flux = [], []
    for lat, F in zip(lats, forces):
        st = LBMState(lat, precision, 20)
        for k in calls:
            st.step(k, WP, WM, F)
        ref_f.append(st.get_pdfs().cpu().numpy())
        ref_flux.append(st.reduce_flux(2) if lat.n > 0 else None)
        st.close()
    for group_bytes in (-1, 1, 3 << 20):
        bs = BatchedState(lats, precision, 20)
        bs.groups(group_bytes)
        n_groups, cap = bs.resident(1)
        assert cap > 0 and n_groups >= 1
        for j, k in enumerate(calls):
            if j == 2:
                bs.resident(0)
            if j == 3:
                bs.resident(1)
            bs.step(k, WP, WM, forces)
        mass, flux = bs.reduce_flux(2)
        f_all = bs.get_pdfs().cpu().numpy()
        for i in range(len(lats)):
            b, c = bs.begin[i], bs.count[i]
            np.testing.assert_array_equal(f_all[:, b:b + c], ref_f[i])
            if ref_flux[i] is not None:
                assert (mass[i], flux[i]) == ref_flux[i]
            else:
                assert (mass[i], flux[i]) == (0.0, 0.0)
        bs.close()
    for lat in lats:
        lat.close()


def test_resident_group_split_and_forms():
    """With resident steps a group's working set is its two PDF grids and a
    group holds at most the resident capacity; FP64 arithmetic is refused."""
    beds, _ = _beds(7, seed=5)
    lats = _lattices(beds)
    bs = BatchedState(lats, "f16s", 20)
    spans = [(c + 2047) // 2048 * 2048 for c in bs.count]
    n1, cap = bs.resident(1)
    per_cell = 2 * 19 * 2
    for budget in (1, 2048 * per_cell, 3 * 2048 * per_cell, 0):
        expect, cur = 0, 0
        for s_ in spans:
            if s_ == 0:
                continue
            if cur > 0 and ((cur + s_) * per_cell > budget or cur + s_ > cap):
                expect += 1
                cur = 0
            cur += s_
        expect += 1
        if budget == 0:
            expect = 1
        assert bs.groups(budget) == expect, budget
    with pytest.raises(capi.LbmError) as ei:
        bs.resident(2)
    assert ei.value.status == capi.LBM_EINVAL
    bs.close()
    for precision in ("f64", "f64x"):
        bs = BatchedState(lats, precision, 0)
        with pytest.raises(capi.LbmError) as ei:
            bs.resident(1)
        assert ei.value.status == capi.LBM_EINVAL
        bs.close()
    for lat in lats:
        lat.close()


def test_resident_barrier_time_limit_reports_and_recovers():
    """Check mode: every barrier wait expects one block more than the grid
    holds, so each resident launch gives up after its 20 ms limit; the call
    is reported as LBM_ETIMEOUT by lbm_reduce_flux, the flag clears, and the
    state then steps correctly from a reset."""
    beds, forces = _beds(4, seed=6)
    lats = _lattices(beds)
    bs = BatchedState(lats, "f32s", 0)
    bs.groups(1)
    bs.resident(-1)
    bs.step(4, WP, WM, forces)
    with pytest.raises(capi.LbmError) as ei:
        bs.reduce_flux(2)
    assert ei.value.status == capi.LBM_ETIMEOUT
    bs.resident(1)
    bs.reset()
    bs.step(6, WP, WM, forces)
    mass, flux = bs.reduce_flux(2)
    for i, lat in enumerate(lats):
        if lat.n == 0:
            continue
        st = LBMState(lat, "f32s", 0)
        st.step(6, WP, WM, forces[i])
        assert st.reduce_flux(2) == (mass[i], flux[i])
        st.close()
    bs.close()
    for lat in lats:
        lat.close()


def test_resident_mode_steps_a_bed_above_the_capacity_per_step():
    """A bed larger than the resident capacity forms a group of its own and
    keeps the per-step launches; the small beds beside it run resident.
    Both stay bit-identical to their separate runs."""
    big = inputs.packed_bed((128, 128, 128), 2, 126.0, 6.0, 0.45, 11)
    beds, forces = _beds(3, seed=7)
    beds = [beds[0], big] + beds[1:]
    forces = [forces[0], (2e-6, 0.0, 1e-6)] + forces[1:]
    lats = _lattices(beds)
    bs = BatchedState(lats, "f16s", 20)
    n_groups, cap = bs.resident(1)
    assert lats[1].n > cap and n_groups >= 3
    bs.step(5, WP, WM, forces)
    mass, flux = bs.reduce_flux(2)
    f_all = bs.get_pdfs().cpu().numpy()
    for i, (lat, F) in enumerate(zip(lats, forces)):
        if lat.n == 0:
            continue
        st = LBMState(lat, "f16s", 20)
        st.step(5, WP, WM, F)
        b, c = bs.begin[i], bs.count[i]
        np.testing.assert_array_equal(f_all[:, b:b + c], st.get_pdfs().cpu().numpy())
        assert st.reduce_flux(2) == (mass[i], flux[i])
        st.close()
    bs.close()
    for lat in lats:
        lat.close()
