"""The index-range limits of the int32 adjacency, at full size.

A state's PDF slot is addressed as q*L + m in int32, L the row stride (N
rounded up to 64), so the library accepts at most 19*L < 2^31 (N <=
113,025,408).  All-fluid periodic boxes just below that limit are assembled
and stepped in the FP64-storage form: 1024 x 512 x 215 = 112,721,920 cells
(L = N, the last PDF slot at 2,141,716,479) and 1023 x 511 x 215 =
112,391,895 cells (rows padded to L = 112,391,936, the last slot at
2,135,446,783), in the FP64-storage form and in FP16 shifted storage (whose
first step runs the pair sweep).  Every cell sees the same history, so
every cell's moments must be identical and equal those of a single periodic
cell stepped by the oracle (to FP64 round-off, or to FP16 storage), and the
mass must stay N.  Any index that wrapped past 2^31 would break that
uniformity.  A slightly larger all-fluid box (1024 x 512 x 256, 19*N =
2.55e9) must be refused with LBM_EOVERFLOW before any PDF or adjacency
memory is taken.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1111_1129_gb300 import (LBMState, SparseLattice, build, capi, omega_minus,
                                   shifted_scale_exp)

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (3e-6, -1e-6, 2e-6)


@pytest.fixture(scope="module", autouse=True)
def library():
    build.build()
    capi.load()


@pytest.mark.parametrize("precision", ["f64x", "f16s"])
@pytest.mark.parametrize("dims", [(1024, 512, 215), (1023, 511, 215)])   # x, y, z
def test_largest_list_steps_uniformly(dims, precision):
    """FP64 storage (the fixed-point sweep) and FP16 shifted (the pair sweep
    for the first step, whose rest row is read as 32-bit words and whose
    stores are paired): every cell must leave the two steps identical."""
    n_box = dims[0] * dims[1] * dims[2]
    ld = -(-n_box // 64) * 64
    assert 19 * ld < 2 ** 31 <= 19 * 1024 * 512 * 216
    assert (ld == n_box) == (dims[0] == 1024)
    flags = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.uint8, device="cuda")
    lat = SparseLattice(flags, "lex", periodic=0b111)
    del flags
    assert lat.n == n_box
    k = shifted_scale_exp(1e-5) if precision == "f16s" else 0
    st = LBMState(lat, precision, k)
    st.step(2, WP, WM, F)
    mass, flux = st.reduce_flux(0)
    rho, u = st.moments()
    # one periodic cell, two steps, in the oracle
    one = np.zeros((1, 1, 1), np.uint8)
    _, obs, rho1, u1 = oracle.run(one, 0b111, WP, WM, F, 2)
    # f64x: u ~ 1e-6 is a sum of +-f ~ 0.03, FP64 round-off of the sums is
    # ~1e-17 absolute, ~1e-11 relative, and the two sides sum in different
    # orders.  FP16: deviations ~1e-6 stored to 11 bits.
    rel = 1e-10 if precision == "f64x" else 2e-3
    if precision == "f64x":
        assert mass == float(n_box)                 # rest + force: rho = 1 exactly
    else:
        assert abs(mass - n_box) <= 1e-9 * n_box
    assert abs(flux - u1[0, 0, 0, 0]) <= rel * abs(u1[0, 0, 0, 0])
    for d in range(3):
        col = u[d]
        assert torch.equal(col, col[:1].expand_as(col)), d   # every cell identical
        assert abs(float(col[0]) - u1[d, 0, 0, 0]) <= rel * abs(u1[d, 0, 0, 0])
    assert torch.equal(rho, rho[:1].expand_as(rho))
    assert abs(float(rho[0]) - rho1[0, 0, 0]) <= (1e-15 if precision == "f64x" else 1e-9)
    del rho, u
    st.close()
    lat.close()


def test_list_beyond_the_slot_range_is_refused():
    dims = (1024, 512, 256)
    flags = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.LbmError) as ei:
        SparseLattice(flags, "lex", periodic=0b111)
    assert ei.value.status == capi.LBM_EOVERFLOW
    assert "19*L" in str(ei.value)
