"""lbm_set_allocator: with PyTorch's caching allocator behind the library,
every handle's device memory shows in torch.cuda.memory_allocated() and goes
back when the handle is freed, the allocator cannot change while handles
are alive, and results equal those with the library's own allocator bit for
bit (single bed, batched beds in L2 groups, adjoint)."""
import pytest
import torch

from paper_1111_1129_gb300 import (Adjoint, BatchedState, LBMState, SparseLattice, build, capi,
                                   inputs, omega_minus, use_torch_allocator)

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (0.0, 0.0, 1e-5)


def _run(flags, periodic):
    lat = SparseLattice(flags, "lex", (8, 8, 8), periodic)
    st = LBMState(lat, "f64x")
    st.step(40, WP, WM, F)
    out = [st.get_pdfs().cpu(), st.reduce_flux(2)]
    st.close()
    beds = [SparseLattice(flags, "lex", (8, 8, 8), periodic) for _ in range(3)]
    bs = BatchedState(beds, "f32s")
    bs.groups(1)   # every bed its own group: regrouping allocates and frees
    bs.step(30, WP, WM, [F, (0.0, 0.0, 2e-5), (1e-6, 0.0, 0.0)])
    out += [bs.get_pdfs().cpu(), bs.reduce_flux(2)]
    bs.close()
    for b in beds:
        b.close()
    st = LBMState(lat, "f32s")
    ad = Adjoint(st, 12, 4)
    out.append(ad.forward(WP, WM, F, 2))
    out.append(ad.backward()[0])
    ad.close()
    st.close()
    lat.close()
    return out


def test_torch_allocator_holds_and_returns_the_memory():
    build.build()
    capi.load()
    bed = inputs.bed_small(0)
    flags = torch.from_numpy(bed.flags).cuda()
    ref = _run(flags, bed.periodic)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    use_torch_allocator(True)
    try:
        lat = SparseLattice(flags, "lex", (8, 8, 8), bed.periodic)
        st = LBMState(lat, "f64x")
        held = torch.cuda.memory_allocated() - before
        assert held >= 2 * 19 * 8 * lat.n + 18 * 4 * lat.n, held
        with pytest.raises(RuntimeError, match="still live"):
            capi.lbm_set_allocator(None, None)
        st.close()
        lat.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        got = _run(flags, bed.periodic)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        use_torch_allocator(False)
    assert torch.equal(ref[0], got[0]) and ref[1] == got[1]
    assert torch.equal(ref[2], got[2])
    assert list(ref[3][0]) == list(got[3][0]) and list(ref[3][1]) == list(got[3][1])
    assert ref[4] == got[4] and list(ref[5]) == list(got[5])
