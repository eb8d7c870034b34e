"""The allocation-free FP64 step (lbm_step_f64_noalloc), for callers that
cannot allocate device memory -- for example an application that owns all
of the GPU's memory and lends this library only the arrays it works on.

Its output must equal what the allocating entry points produce (lbm_step on
an FP64 state, then lbm_state_get_pdfs and lbm_reduce_flux along each axis)
within the FP64 tolerance of the other tests, on two calls in a row.  After
a first call on the device (which loads the library's code there and with
it the static scratch), further calls must leave the device's free memory
unchanged.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


@pytest.mark.parametrize("damped", [False, True])
def test_noalloc_step_matches_the_allocating_entry_points(damped):
    bed = inputs.bed_small(3)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "blocked", (8, 8, 8), bed.periodic)
    n, _, adj_ptr, _ = capi.lbm_sparse_info(lat.handle)
    st = LBMState(lat, "f64")
    rng = np.random.default_rng(4)
    w = st.get_pdfs()[:, :1].cpu().numpy()
    f0 = torch.from_numpy(w * (1.0 + 0.01 * rng.standard_normal((19, n)))).cuda()
    st.set_pdfs(f0)
    alpha = None
    if damped:
        alpha = torch.from_numpy(0.05 * rng.random(n)).cuda()
        st.set_damping(alpha)
    F = (1e-5, -2e-6, 3e-5)
    fa = f0.clone()
    fb = torch.empty_like(fa)
    warm = torch.empty_like(fa)
    sums = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    a_ptr = alpha.data_ptr() if damped else None
    # first call on the device: loads the code and its static scratch
    capi.lbm_step_f64_noalloc(fa.data_ptr(), warm.data_ptr(), adj_ptr, n, WP, WM, F, a_ptr,
                              sums.data_ptr(), stream)
    torch.cuda.synchronize()
    for _ in range(2):
        st.step(1, WP, WM, F)
        ref_sums = [st.reduce_flux(axis) for axis in range(3)]
        ref = st.get_pdfs()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        capi.lbm_step_f64_noalloc(fa.data_ptr(), fb.data_ptr(), adj_ptr, n, WP, WM, F, a_ptr,
                                  sums.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        err = (fb - ref).abs().max().item() / ref.abs().max().item()
        assert err <= TOL, err
        s = sums.cpu().numpy()
        mass = ref_sums[0][0]
        assert abs(s[0] - mass) <= TOL * abs(mass)
        for axis in range(3):
            flux = ref_sums[axis][1]
            assert abs(s[1 + axis] / n - flux) <= TOL * max(abs(flux), 1e-300), (axis, s, flux)
        fa, fb = fb, fa
    st.close()
    lat.close()


def test_noalloc_step_rejects_sizes_beyond_its_scratch():
    sums = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.LbmError) as ei:
        capi.lbm_step_f64_noalloc(0, 0, 0, 16_777_217, WP, WM, (0, 0, 0), None,
                                  sums.data_ptr(), 0)
    assert ei.value.status == capi.LBM_EINVAL
    assert "16777216" in str(ei.value)


def test_noalloc_step_on_an_empty_list_gives_zero_sums():
    sums = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    capi.lbm_step_f64_noalloc(0, 0, 0, 0, WP, WM, (0.0, 0.0, 1e-6), None, sums.data_ptr(),
                              stream)
    torch.cuda.synchronize()
    assert sums.tolist() == [0.0, 0.0, 0.0, 0.0]
