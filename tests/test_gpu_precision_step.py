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

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)
F = (3e-6, -2e-6, 5e-6)
DEV = 1e-4
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lattice():
    build.build()
    capi.load()
    bed = inputs.bed_small(1)
    cells, _, adj = oracle.build_sparse(bed.flags, oracle.ORDER_LEX, periodic=bed.periodic)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", periodic=bed.periodic)
    np.testing.assert_array_equal(lat.cells().cpu().numpy(), cells)
    yield lat, adj, len(cells)
    lat.close()


def _ulp_f16(v):
    """Spacing of FP16 at |v| (v already scaled), from numpy's float16."""
    return np.spacing(np.abs(v).astype(np.float16)).astype(np.float64)


def _ulp_bf16(v):
    """Spacing of BF16 (8-bit significand, FP32 exponent range) at |v|."""
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 2.0 ** -126)))
    return 2.0 ** (np.maximum(e, -126) - 7)


def _ulp_f32(v):
    return np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)


def _rn_bf16(v):
    """Round FP64 to BF16 (via FP32, nearest even), returned as FP64."""
    u = np.asarray(v, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


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

    dev_rep = f_rep - W[:, None]
    big = 19.0 * np.abs(dev_rep).max()         # bound on any intermediate deviation sum
    err = np.abs(f_gpu - f_ref)
    scale = 2.0 ** k
    d_ref = (f_ref - W[:, None]) * scale        # exact: the subtraction cancels w's bits
    if precision == "f16s":
        tol = _ulp_f16(d_ref) / scale + 64 * EPS32 * big
    elif precision == "bf16s":
        tol = _ulp_bf16(d_ref) / scale + 64 * EPS32 * big
    elif precision == "f32s":   # measured: 0.14 of this bound
        tol = _ulp_f32(f_ref - W[:, None]) + 4 * EPS32 * big
    else:   # FP32 of f itself: the arithmetic works on values up to rho ~ 1 (measured 0.27)
        tol = _ulp_f32(f_ref) + 6 * EPS32
    worst = float((err / tol).max())
    print(f"{precision} damped={damped} n={n} k={k} max|err|={err.max():.3e} "
          f"max err/tol={worst:.3f}")
    assert np.isfinite(f_gpu).all()
    assert worst <= 1.0, (precision, damped, worst)

    if precision in ("f16s", "bf16s"):
        code_gpu = (f_gpu - W[:, None]) * scale
        code_ref = (d_ref.astype(np.float16).astype(np.float64) if precision == "f16s"
                    else _rn_bf16(d_ref))
        same = float(np.mean(code_gpu == code_ref))
        print(f"{precision} damped={damped}: codes equal to the rounded FP64 result: {same:.5f}")
        assert same >= 0.99, same
