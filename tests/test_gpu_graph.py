"""lbm_step replays a cached CUDA graph of non-reducing steps for long calls.

The graph holds the same kernels, in the same order, as the launches it
replaces, so a run stepped in long calls (graph replays) must equal the same
run stepped in short calls (individual launches) bit for bit, in PDFs and in
the reduced mass and flux.  The cases cover both grid parities (odd step
counts), a change of force and of relaxation rates between calls (the graph
must be recaptured), and damping switched on after a graph was captured.
"""
import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)


@pytest.fixture(scope="module")
def lattice():
    build.build()
    capi.load()
    bed = inputs.bed_small(3)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "blocked", (8, 8, 8), bed.periodic)
    yield lat
    lat.close()


def _run(lat, precision, plan, chunk, alpha_at=None):
    """Run `plan` = [(steps, omega_plus, force), ...]; every call is split
    into calls of at most `chunk` steps (chunk=None: one call each)."""
    st = LBMState(lat, precision, 22)
    rng = np.random.default_rng(5)
    alpha = torch.from_numpy(rng.uniform(0.0, 0.05, lat.n))
    flux = []
    for j, (steps, wp, F) in enumerate(plan):
        if alpha_at is not None and j == alpha_at:
            st.set_damping(alpha)
        left = steps
        while left > 0:
            k = left if chunk is None else min(chunk, left)
            st.step(k, wp, omega_minus(wp), F)
            left -= k
        flux.append(st.reduce_flux(2))
    f = st.get_pdfs()
    st.close()
    return f, flux


@pytest.mark.parametrize("precision", ["f64x", "f64", "f32s", "f16s"])
def test_long_calls_equal_short_calls(lattice, precision):
    plan = [(1000, WP, (0.0, 0.0, 1e-5)), (301, WP, (0.0, 0.0, 1e-5)),
            (300, WP, (0.0, 0.0, 1e-5))]
    f_graph, flux_graph = _run(lattice, precision, plan, None)
    f_plain, flux_plain = _run(lattice, precision, plan, 7)
    assert torch.equal(f_graph, f_plain)
    assert flux_graph == flux_plain


@pytest.mark.parametrize("precision", ["f64x", "f32s"])
def test_changed_arguments_recapture(lattice, precision):
    plan = [(400, WP, (0.0, 0.0, 1e-5)), (400, WP, (2e-6, 0.0, 3e-5)),
            (401, 1.5, (2e-6, 0.0, 3e-5)), (400, 1.5, (2e-6, 0.0, 3e-5))]
    f_graph, flux_graph = _run(lattice, precision, plan, None, alpha_at=3)
    f_plain, flux_plain = _run(lattice, precision, plan, 9, alpha_at=3)
    assert torch.equal(f_graph, f_plain)
    assert flux_graph == flux_plain
