"""Chained steps: within one lbm_step call the second and later sweeps are
launched with programmatic dependent launch, so a sweep's blocks can start
before the previous sweep has finished and wait inside the kernel.  A run in
one call must therefore equal the same run taken one step per call (where no
launch is chained) bit for bit, in PDFs and in the reduced sums.  The cases
cover every storage form, with and without damping, a bed of one wave (whose
FP32 and 16-bit sweeps load their links before the wait) and a bed of many
waves.
"""
import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (0.0, 0.0, 1e-5)
STEPS = 41


@pytest.fixture(scope="module", params=["one_wave", "many_waves"])
def lattice(request):
    build.build()
    capi.load()
    bed = inputs.bed_small(1) if request.param == "one_wave" else inputs.bed_cube128(2)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", (8, 8, 8), bed.periodic)
    yield lat
    lat.close()


def _run(lat, precision, damped, calls):
    st = LBMState(lat, precision, 22)
    if damped:
        rng = np.random.default_rng(9)
        st.set_damping(torch.from_numpy(rng.uniform(0.0, 0.05, lat.n)))
    for n in calls:
        st.step(n, WP, WM, F)
    out = st.get_pdfs(), st.reduce_flux(2)
    st.close()
    return out


@pytest.mark.parametrize("damped", [False, True])
@pytest.mark.parametrize("precision", ["f64x", "f64", "f32", "f32s", "f16s", "bf16s"])
def test_one_call_equals_single_steps(lattice, precision, damped):
    f_one, sums_one = _run(lattice, precision, damped, [STEPS])
    f_single, sums_single = _run(lattice, precision, damped, [1] * STEPS)
    assert torch.equal(f_one, f_single)
    assert sums_one == sums_single
