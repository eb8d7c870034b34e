"""lbm_step_timed: the device time of a call's steps from CUDA events on the
state's stream, with the same results as lbm_step."""
import ctypes

import pytest
import torch

from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (1e-6, 0.0, 0.0)


def test_timed_steps_match_plain_steps_and_events():
    build.build()
    capi.load()
    bed = inputs.bed_medium(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", (8, 8, 8), bed.periodic)
    a, b = LBMState(lat, "f64x"), LBMState(lat, "f64x")
    a.step(40, WP, WM, F)
    ms = b.step_timed(40, WP, WM, F)
    assert torch.equal(a.get_pdfs(), b.get_pdfs())
    assert a.reduce_flux(0) == b.reduce_flux(0)
    # the same work timed with torch's events on the same stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    a.step(40, WP, WM, F)
    e1.record()
    torch.cuda.synchronize()
    ref = e0.elapsed_time(e1)
    assert ms > 0 and 0.5 * ref < ms < 2.0 * ref, (ms, ref)
    lib = capi.load()
    f = (ctypes.c_double * 3)(*F)
    assert lib.lbm_step_timed(b.handle, 1, WP, WM, f, None) == capi.LBM_EINVAL
    a.close()
    b.close()
    lat.close()
