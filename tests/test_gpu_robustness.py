"""Checkpoint/resume and failure detection, with every failure made on the
host side (no fault, trap or hang on the GPU): a wait that runs out of
time returns LBM_ETIMEOUT and the context stays usable; a non-finite state
is reported by the reduction; a resumed run continues bit for bit."""
import numpy as np
import pytest
import torch

from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


@pytest.mark.parametrize("force", [1e-5, 1e-9])
@pytest.mark.parametrize("precision", ["f64", "f64x", "f32", "f32s", "f16s", "bf16s"])
def test_checkpoint_resume_is_bit_exact(precision, force, tmp_path):
    """A checkpoint holds the stored words, so a resumed run continues bit
    for bit.  At F = 1e-9 most FP32 deviations after 30 steps are far below
    1e-9, where w + d in FP64 no longer carries d: a checkpoint of FP64 PDFs
    could not restore them."""
    bed = inputs.bed_small(4)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "morton1", periodic=bed.periodic)
    F = (0.0, 0.0, force)
    a = LBMState(lat, precision, 22)
    a.step(30, WP, WM, F)
    a.save(str(tmp_path / "ck.npz"), force=F)
    a.step(25, WP, WM, F)
    ref = a.get_pdfs()
    ref_flux = a.reduce_flux(2)
    b = LBMState(lat, precision, 22)
    meta = b.load(str(tmp_path / "ck.npz"))
    assert tuple(meta["force"]) == F and int(meta["steps"]) == 30
    b.step(25, WP, WM, F)
    assert torch.equal(b.get_pdfs(), ref)
    assert b.reduce_flux(2) == ref_flux
    other = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    with pytest.raises(ValueError):
        LBMState(other, precision, 22).load(str(tmp_path / "ck.npz"))
    for h in (a, b, other, lat):
        h.close()


@pytest.mark.parametrize("precision", ["f64x", "f32s", "f16s"])
def test_raw_copies_round_trip_exactly(precision):
    """lbm_state_get_raw / set_raw copy the stored words ([19][N], the
    state's padded rows removed), to device and to pageable host memory."""
    bed = inputs.bed_small(2)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    assert lat.n % 64 != 0                      # the state's rows are padded
    F = (0.0, 0.0, 1e-7)
    a = LBMState(lat, precision, 24)
    a.step(17, WP, WM, F)
    raw = a.get_raw()
    b = LBMState(lat, precision, 24)
    b.set_raw(raw)
    assert torch.equal(b.get_raw(), raw) and torch.equal(b.get_pdfs(), a.get_pdfs())
    host = np.zeros(tuple(raw.shape), dtype=raw.cpu().numpy().dtype)      # pageable
    capi.lbm_state_get_raw(a.handle, host.ctypes.data)
    np.testing.assert_array_equal(host, raw.cpu().numpy())
    c = LBMState(lat, precision, 24)
    capi.lbm_state_set_raw(c.handle, host.ctypes.data)
    a.step(3, WP, WM, F)
    c.step(3, WP, WM, F)
    assert torch.equal(c.get_raw(), a.get_raw())
    with pytest.raises(ValueError):
        c.set_raw(raw[:, :-1])
    for fn in (capi.lbm_state_get_raw, capi.lbm_state_set_raw):
        with pytest.raises(capi.LbmError) as ei:
            fn(c.handle, None)
        assert ei.value.status == capi.LBM_EINVAL
    for h in (a, b, c, lat):
        h.close()
    # an empty list: nothing to copy, no pointer needed
    empty = SparseLattice(torch.ones((3, 4, 5), dtype=torch.uint8).cuda(), "lex")
    st = LBMState(empty, precision, 24)
    capi.lbm_state_get_raw(st.handle, None)
    capi.lbm_state_set_raw(st.handle, None)
    assert st.get_raw().shape == (19, 0)
    st.close()
    empty.close()


def test_wait_with_a_time_limit_reports_timeout_and_recovers():
    bed = inputs.bed_medium(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "blocked", (8, 8, 8), bed.periodic)
    st = LBMState(lat, "f64")                  # IEEE FP64: ~0.5 ms per step here
    st.step(2000, WP, WM, (1e-6, 0.0, 0.0))    # ~1 s of queued work
    with pytest.raises(capi.LbmError) as ei:
        st.synchronize(1e-3)
    assert ei.value.status == capi.LBM_ETIMEOUT
    st.synchronize(600.0)                      # the same work completes normally
    capi.lbm_set_timeout(1e-3)
    try:
        st.step(2000, WP, WM, (1e-6, 0.0, 0.0))
        with pytest.raises(capi.LbmError) as ei:
            st.reduce_flux(0)
        assert ei.value.status == capi.LBM_ETIMEOUT
    finally:
        capi.lbm_set_timeout(600.0)
    mass, flux = st.reduce_flux(0)
    assert abs(mass - lat.n) < 1e-9 * lat.n and flux > 0
    st.close()
    lat.close()


@pytest.mark.parametrize("precision", ["f64", "f64x", "f32s", "f16s"])
def test_non_finite_state_is_reported(precision):
    """A NaN must survive the reduction's fixed-point warp sums (the warp
    holding it sums in FP64) and be reported."""
    bed = inputs.bed_small(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    st = LBMState(lat, precision, 22)
    f = st.get_pdfs()
    f[3, 17] = float("nan")
    st.set_pdfs(f)
    st.step(2, WP, WM, (0.0, 0.0, 1e-6))
    with pytest.raises(capi.LbmError) as ei:
        st.reduce_flux(2)
    assert ei.value.status == capi.LBM_ENONFINITE
    st.close()
    lat.close()


def test_errors_leave_a_readable_message_per_thread():
    with pytest.raises(capi.LbmError):
        capi.lbm_state_create(0, 0, 0)
    assert "sparse" in capi.lbm_last_error()
    import threading
    seen = []
    t = threading.Thread(target=lambda: seen.append(capi.lbm_last_error()))
    t.start()
    t.join()
    assert seen == [""]


def test_allocation_failure_is_reported_and_leaves_the_state_usable():
    """An adjoint whose checkpoints would need petabytes: the device refuses
    the allocation at once (nothing is consumed), the call returns
    LBM_ENOMEM with a message, and the state steps on normally."""
    bed = inputs.bed_small(0)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    st = LBMState(lat, "f64")
    with pytest.raises(capi.LbmError) as ei:
        capi.lbm_adjoint_create(st.handle, 2 ** 31 - 1, 1)
    assert ei.value.status == capi.LBM_ENOMEM
    assert "checkpoints" in str(ei.value)
    st.step(10, WP, WM, (0.0, 0.0, 1e-6))
    mass, flux = st.reduce_flux(2)
    assert abs(mass - lat.n) < 1e-12 * lat.n and flux > 0
    st.close()
    lat.close()
