"""One step of each reduced storage form against the FP64 oracle, to the
storage unit.

The steady-state test bounds the accumulated error of the precision forms;
this one pins a single update.  A random non-equilibrium state (deviations
f - w up to 1e-4, a force with all three components, with and without
Brinkman damping) is written into the state, read back -- what the form
actually stores, decoded exactly to FP64 -- and stepped once on the GPU and
once by the oracle's sparse stepper from that same read-back state.

The GPU computes in FP32 and rounds once into storage, so every output must
lie within one storage unit of the FP64 result, plus the FP32 rounding of
the collision: 4 x 2^-24 of the largest intermediate deviation sum for the
shifted forms, 6 x 2^-24 (of rho ~ 1) for FP32 of f itself.  For the
16-bit forms the stored code must also equal the FP64 result rounded to
nearest even at the same scale, except where the FP32 arithmetic lands on
the other side of a rounding midpoint: at most 1% of the codes.

The reading of the storage forms (deviation from w_q, scaled by 2^k, round
to nearest) is the one the steady-state test and the kernels share (the
paper stores FP64 and names no reduced form).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1111_1129_gb300 import LBMState, SparseLattice, build, capi, inputs, omega_minus
from paper_1111_1129_gb300 import shifted_scale_exp
from storage_units import W, codes_equal_fraction, one_step_tolerance

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (3e-6, -2e-6, 5e-6)
DEV = 1e-4


@pytest.fixture(scope="module", params=["ragged", "x64"])
def lattice(request):
    """The small bed (a list whose length is not a multiple of the 64-element
    row alignment, so the state's rows are padded) and the same bed with
    its last fluid cells made solid until the length is one (rows unpadded)."""
    build.build()
    capi.load()
    bed = inputs.bed_small(1)
    flags = bed.flags.copy()
    fluid = np.argwhere(flags == 0)
    assert len(fluid) % 64 != 0
    if request.param == "x64":
        for z, y, x in fluid[len(fluid) - len(fluid) % 64:]:
            flags[z, y, x] = 1
    cells, _, adj = oracle.build_sparse(flags, oracle.ORDER_LEX, periodic=bed.periodic)
    assert (len(cells) % 64 == 0) == (request.param == "x64")
    lat = SparseLattice(torch.from_numpy(flags).cuda(), "lex", periodic=bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    yield lat, adj, len(cells)
    lat.close()


@pytest.mark.parametrize("damped", [False, True])
@pytest.mark.parametrize("precision", ["f16s", "bf16s", "f32s", "f32"])
def test_one_step_within_one_storage_unit(lattice, precision, damped):
    lat, adj, n = lattice
    rng = np.random.default_rng(7 + 2 * damped)
    f0 = W[:, None] + DEV * rng.uniform(-1.0, 1.0, size=(19, n))
    alpha = rng.uniform(0.0, 0.05, size=n) if damped else None
    k = shifted_scale_exp(4 * DEV)   # 4x headroom: a collision can grow a deviation
    assert k <= 33   # keeps w + code * 2^-k exact in FP64 (FP16 subnormals included)
    st = LBMState(lat, precision, k)
    st.set_pdfs(torch.from_numpy(f0))
    if damped:
        st.set_damping(torch.from_numpy(alpha))
    f_rep = st.get_pdfs().cpu().numpy()        # what the form stores, decoded exactly
    st.step(1, WP, WM, F)
    f_gpu = st.get_pdfs().cpu().numpy()
    st.close()
    f_ref = oracle.sparse_step(f_rep, adj, n, F, WP, WM, alpha).reshape(19, n)

    err = np.abs(f_gpu - f_ref)
    tol = one_step_tolerance(precision, f_ref, float(np.abs(f_rep - W[:, None]).max()), k)
    worst = float((err / tol).max())
    print(f"{precision} damped={damped} n={n} k={k} max|err|={err.max():.3e} "
          f"max err/tol={worst:.3f}")
    assert np.isfinite(f_gpu).all()
    assert worst <= 1.0, (precision, damped, worst)

    if precision in ("f16s", "bf16s"):
        same = codes_equal_fraction(precision, f_gpu, f_ref, k)
        print(f"{precision} damped={damped}: codes equal to the rounded FP64 result: {same:.5f}")
        assert same >= 0.99, same
