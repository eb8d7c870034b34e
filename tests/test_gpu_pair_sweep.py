"""The 16-bit sweep that updates two adjacent cells per thread.

Its plain steps run on grids of more than one wave, and the reducing last
step of a call runs the one-cell kernel, so a run taken in one call must
equal the same steps taken one call each bit for bit (same per-cell
arithmetic).  The cases cover both parities of the list length N (an odd
N leaves one cell alone at the end of the list) and an N that needs no
row padding,
damping, and an order in which neighbouring cells rarely pull from
neighbouring slots (Morton, 2-bit) as well as the lexicographic order in
which they mostly do.
"""
import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (2e-6, -1e-6, 1e-5)


@pytest.fixture(scope="module", params=["even", "odd", "x64"])
def flags(request):
    """N even, N odd (rows padded to a multiple of 64 either way), and N a
    multiple of 64 (rows unpadded; the kernels read the plain links)."""
    build.build()
    capi.load()
    bed = inputs.packed_bed((96, 80, 72), 2, 70.0, 5.0, 0.45, 3)
    f = bed.flags.copy()
    fluid = np.argwhere(f == 0)
    mid = len(fluid) // 2
    if request.param == "x64":
        drop = len(fluid) % 64
    else:
        want = 0 if request.param == "even" else 1
        drop = 0 if len(fluid) % 2 == want else 1
        if (len(fluid) - drop) % 64 == 0:
            drop += 2
    for z, y, x in fluid[mid:mid + drop]:
        f[z, y, x] = 1
    n = int((f == 0).sum())
    assert (n % 64 == 0) == (request.param == "x64")
    if request.param != "x64":
        assert n % 2 == (0 if request.param == "even" else 1)
    return f, bed.periodic


@pytest.mark.parametrize("ordering", ["lex", "morton2"])
@pytest.mark.parametrize("damped", [False, True])
@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
def test_pair_steps_equal_single_cell_steps(flags, precision, damped, ordering):
    f, periodic = flags
    lat = SparseLattice(torch.from_numpy(f).cuda(), ordering, (8, 8, 8), periodic)
    assert lat.n > 4 * 152 * 256          # more than one wave: the paired kernel runs
    alpha = None
    if damped:
        alpha = torch.from_numpy(np.random.default_rng(5).uniform(0.0, 0.05, lat.n))
    out = []
    for calls in ([9], [1] * 9):
        st = LBMState(lat, precision, 22)
        if damped:
            st.set_damping(alpha)
        for k in calls:
            st.step(k, WP, WM, F)
        out.append((st.get_pdfs(), st.reduce_flux(2)))
        st.close()
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    lat.close()


@pytest.mark.parametrize("precision", ["f16s", "bf16s", "f32s"])
def test_large_bed_steps_and_one_step_parity(precision):
    """The 1024x256x256 bed at full size in the benchmark's configuration
    (lexicographic order, the 16-bit forms at the benchmark's scale): two
    steps in one call (the pair kernel for the 16-bit forms, then the
    one-cell reducing step) equal two one-step calls (the one-cell kernel
    each) bit for bit, and one step from the stored state matches the
    oracle's collision on 2000 sampled cells within one storage unit."""
    import oracle
    from paper_1111_1129_gb300 import deviation_bound, shifted_scale_exp
    from storage_units import W, one_step_tolerance

    bed = inputs.bed_large(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", (8, 8, 8), bed.periodic)
    assert lat.n > 4 * 152 * 256 and lat.n % 64 != 0   # many waves; padded rows
    F = (1e-6, 0.0, 0.0)
    k = shifted_scale_exp(deviation_bound(F[0], 125.0, WP)) if precision != "f32s" else 0
    # both states reach step 30 by the same launches; a state written with
    # set_pdfs would not do for FP32S, whose round trip through FP64 f is
    # exact in f but not in a deviation below ~1e-9
    a = LBMState(lat, precision, k)
    b = LBMState(lat, precision, k)
    a.step(30, WP, WM, F)
    b.step(30, WP, WM, F)
    f30 = a.get_pdfs()
    assert torch.equal(b.get_pdfs(), f30)
    a.step(2, WP, WM, F)
    b.step(1, WP, WM, F)
    nxt = b.get_pdfs().cpu().numpy()     # one step from f30, for the oracle check
    b.step(1, WP, WM, F)
    assert torch.equal(a.get_pdfs(), b.get_pdfs())
    assert a.reduce_flux(0) == b.reduce_flux(0)
    a.close()
    b.close()
    cells, _, adj = oracle.build_sparse(bed.flags, oracle.ORDER_LEX, periodic=bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    prev = f30.cpu().numpy()
    flat = prev.ravel()
    sample = np.random.default_rng(2).choice(lat.n, 2000, replace=False)
    ref = np.empty((19, sample.size))
    for j, n in enumerate(sample):
        g = np.concatenate([[flat[n]], flat[adj[:, n]]])
        ref[:, j], _, _ = oracle.collide(g, F, 0.0, WP, WM)
    tol = one_step_tolerance(precision, ref, float(np.abs(prev - W[:, None]).max()), k)
    worst = float((np.abs(nxt[:, sample] - ref) / tol).max())
    print(f"large bed {precision} k={k}: one step, 2000 cells, max err/tol {worst:.3f}")
    assert worst <= 1.0
    lat.close()
