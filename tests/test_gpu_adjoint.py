"""GPU adjoint (transposed pull + transposed TRT Jacobian, checkpointed)
against the FP64 CPU oracle's adjoint and against central finite
differences of the GPU FP64 forward path.

Tolerances: FP64 adjoint vs the oracle adjoint 1e-10 relative (norm-wise
for the per-cell fields, whose entries span many decades); FP32 adjoint vs
FP64 finite differences 1e-3 norm-relative over the sampled cells."""
import numpy as np
import pytest
import torch

import oracle
from paper_1111_1129_gb300 import (Adjoint, LBMFlux, LBMState, SparseLattice, build, capi, inputs,
                                   omega_minus)

pytestmark = pytest.mark.gpu

WP = 1.0 / 0.8
WM = omega_minus(WP)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


def _norm_rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _setup(flags, periodic, precision="f64", alpha_dense=None, f0_dense=None, ordering="lex"):
    lat = SparseLattice(torch.from_numpy(flags).cuda(), ordering, (4, 4, 4), periodic)
    st = LBMState(lat, precision)
    cells = lat.cells().cpu().numpy()
    if f0_dense is not None:
        st.set_pdfs(torch.from_numpy(oracle.to_sparse(f0_dense, cells).copy()))
    if alpha_dense is not None:
        st.set_damping(torch.from_numpy(alpha_dense.reshape(-1)[cells].copy()))
    return lat, st, cells


@pytest.mark.parametrize("precision", ["f64", "f64x"])
@pytest.mark.parametrize("shape,periodic,K,stride", [
    ((4, 5, 6), 0b100, 1, 0), ((4, 5, 6), 0b100, 6, 2), ((5, 4, 3), 0b011, 9, 0),
    ((3, 3, 3), 0b111, 5, 1), ((6, 4, 5), 0b000, 12, 5), ((2, 7, 4), 0b010, 7, 7)])
def test_fp64_adjoint_matches_oracle_adjoint(shape, periodic, K, stride, precision):
    """FP64 arithmetic (IEEE) and FP64 storage whose steps run in fixed
    point, damped, against the oracle's explicit-Jacobian adjoint."""
    rng = np.random.default_rng(sum(shape) * 31 + K)
    flags = (rng.random(shape) < 0.25).astype(np.uint8)
    alpha = 0.05 * rng.random(shape)
    F = np.array([1e-4, -2e-4, 1e-3])
    f0 = oracle.rest_state(flags) * (1 + 0.01 * rng.standard_normal((19,) + shape))
    axis = 2
    J_ref, dF_ref, da_ref, lam0_ref = oracle.adjoint(flags, periodic, WP, WM, F, K, axis,
                                                     alpha=alpha, f0=f0)
    lat, st, cells = _setup(flags, periodic, precision, alpha_dense=alpha, f0_dense=f0)
    adj = Adjoint(st, K, stride)
    J = adj.forward(WP, WM, F, axis)
    dF, da, df0 = adj.backward(want_alpha=True, want_f0=True)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    assert _norm_rel(dF, dF_ref) <= 1e-10
    assert _norm_rel(da.cpu().numpy(), oracle.to_sparse(da_ref, cells)) <= 1e-10
    assert _norm_rel(df0.cpu().numpy(), oracle.to_sparse(lam0_ref, cells)) <= 1e-10
    # backward is repeatable (it recomputes from the checkpoints)
    dF2, da2, _ = adj.backward()
    assert dF2 == dF
    assert torch.equal(da2, da)
    adj.close()
    st.close()
    lat.close()


@pytest.mark.parametrize("precision", ["f64", "f64x"])
def test_fp64_adjoint_with_strong_damping_matches_oracle(precision):
    """Damping drawn in [0, 1]: the FP64-storage form's cells with
    alpha >= 1/2 take the IEEE paths of the fixed-point sweep and of the
    double-single reverse step, the others the fast paths."""
    rng = np.random.default_rng(77)
    shape = (6, 5, 7)
    flags = (rng.random(shape) < 0.2).astype(np.uint8)
    alpha = rng.random(shape)
    F = np.array([2e-4, 1e-4, -5e-4])
    f0 = oracle.rest_state(flags) * (1 + 0.005 * rng.standard_normal((19,) + shape))
    K, axis = 8, 0
    J_ref, dF_ref, da_ref, lam0_ref = oracle.adjoint(flags, 0b001, WP, WM, F, K, axis,
                                                     alpha=alpha, f0=f0)
    lat, st, cells = _setup(flags, 0b001, precision, alpha_dense=alpha, f0_dense=f0)
    assert (oracle.to_sparse(alpha, cells) >= 0.5).any()
    adj = Adjoint(st, K, 3)
    J = adj.forward(WP, WM, F, axis)
    dF, da, df0 = adj.backward(want_alpha=True, want_f0=True)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    assert _norm_rel(dF, dF_ref) <= 1e-10
    assert _norm_rel(da.cpu().numpy(), oracle.to_sparse(da_ref, cells)) <= 1e-10
    assert _norm_rel(df0.cpu().numpy(), oracle.to_sparse(lam0_ref, cells)) <= 1e-10
    adj.close()
    st.close()
    lat.close()


@pytest.mark.parametrize("precision", ["f64", "f64x", "f32s"])
def test_checkpoint_stride_does_not_change_the_result(precision):
    bed = inputs.packed_bed((20, 18, 24), 2, 16.0, 3.0, 0.45, 3)
    alpha = inputs.alpha_field(bed.dims, seed=3)
    lat, st, _ = _setup(bed.flags, bed.periodic, precision, alpha_dense=alpha,
                        ordering="morton1")
    ref = None
    for stride in (1, 3, 7, 30, 40):
        adj = Adjoint(st, 40, stride)
        J = adj.forward(WP, WM, (0.0, 0.0, 1e-5), 2)
        dF, da, _ = adj.backward()
        got = (J, dF, da.cpu().numpy())
        if ref is None:
            ref = got
        else:
            assert got[0] == ref[0] and got[1] == ref[1]
            np.testing.assert_array_equal(got[2], ref[2])
        adj.close()
    st.close()
    lat.close()


def test_autograd_function_matches_finite_differences():
    bed = inputs.packed_bed((16, 16, 20), 2, 14.0, 3.0, 0.45, 4)
    lat, st, cells = _setup(bed.flags, bed.periodic)
    rng = np.random.default_rng(5)
    alpha = torch.tensor(0.05 * rng.random(lat.n), dtype=torch.float64, device="cuda",
                         requires_grad=True)
    force = torch.tensor([0.0, 0.0, 1e-5], dtype=torch.float64, requires_grad=True)
    K = 30
    adj = Adjoint(st, K)
    J = LBMFlux.apply(force, alpha, adj, WP, WM, 2)
    J.backward()

    def J_of(F, a):
        st.set_damping(a)
        return adj.forward(WP, WM, F, 2)

    h = 1e-7
    fd = (J_of([0, 0, 1e-5 + h], alpha.detach()) - J_of([0, 0, 1e-5 - h], alpha.detach())) / (2 * h)
    assert abs(force.grad[2].item() - fd) <= 1e-7 * abs(fd)
    # h = 1e-4: central-difference truncation ~3e-9 relative here, while a
    # smaller h lets the ~1e-14 relative rounding noise of J dominate
    for n in rng.choice(lat.n, 5, replace=False):
        ap, am = alpha.detach().clone(), alpha.detach().clone()
        ap[n] += 1e-4
        am[n] -= 1e-4
        fd = (J_of([0, 0, 1e-5], ap) - J_of([0, 0, 1e-5], am)) / 2e-4
        assert abs(alpha.grad[n].item() - fd) <= 1e-6 * abs(fd) + 1e-16
    adj.close()
    st.close()
    lat.close()


def test_fp32_adjoint_on_128cube_bed_against_fd():
    """The 128^3 bed (tube D=126, r=6 spheres, damping uniform in
    [0, 0.05)), FP32 storage and arithmetic, K = 2000, checkpoints every
    45 steps: dJ/dalpha at 64 seeded random fluid cells and dJ/dF_z against
    central differences (h = 1e-4) of the FP64 forward path."""
    bed = inputs.bed_cube128(0)
    alpha_dense = inputs.alpha_field(bed.dims, seed=0)
    K, F = 2000, (0.0, 0.0, 1e-6)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "blocked", (8, 8, 8), bed.periodic)
    cells = lat.cells().cpu().numpy()
    alpha = torch.from_numpy(alpha_dense.reshape(-1)[cells].copy()).cuda()
    st32 = LBMState(lat, "f32s")
    st32.set_damping(alpha)
    adj = Adjoint(st32, K, 45)
    J32 = adj.forward(WP, WM, F, 2)
    dF, da, _ = adj.backward()
    da = da.cpu().numpy()
    st64 = LBMState(lat, "f64")

    def J64(Fz, a):
        st64.set_pdfs(torch.from_numpy(np.repeat(oracle.velocity_set()[1][:, None], lat.n, 1)))
        st64.set_damping(a)
        st64.step(K, WP, WM, (0.0, 0.0, Fz))
        return st64.reduce_flux(2)[1]

    J = J64(F[2], alpha)
    assert abs(J32 - J) <= 1e-5 * abs(J)
    h = 1e-4
    rng = np.random.default_rng(0)
    sample = rng.choice(lat.n, 64, replace=False)
    fd = []
    for n in sample:
        ap, am = alpha.clone(), alpha.clone()
        ap[n] += h
        am[n] -= h
        fd.append((J64(F[2], ap) - J64(F[2], am)) / (2 * h))
    err = _norm_rel(da[sample], fd)
    assert err <= 1e-3, err
    hF = 1e-4 * F[2]
    fdF = (J64(F[2] + hF, alpha) - J64(F[2] - hF, alpha)) / (2 * hF)
    assert abs(dF[2] - fdF) <= 1e-3 * abs(fdF)
    adj.close()
    st32.close()
    st64.close()
    lat.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f64x", 1e-10)])
@pytest.mark.parametrize("K", [2, 3])
def test_fp64_adjoint_equals_exact_directional_derivatives_on_the_128cube_bed(precision, tol, K):
    """The dot-product test at full scale, on the damped 128^3 bed (1.03 M
    cells).  One step is a quadratic polynomial of the state and of F, so J
    after K = 2 steps is quadratic along any direction v of f0 and in F: the
    central difference of the GPU's own forward path is the exact
    derivative.  After K = 3 steps J is quartic, and (4 D(h) - D(2h)) / 3
    is exact.  <dJ/df0, v> and dJ/dF of the GPU adjoint must match these to
    round-off: tol, relative (the FP64-storage adjoint reverses in
    double-single arithmetic, ~48 bits)."""
    bed = inputs.bed_cube128(0)
    alpha_dense = inputs.alpha_field(bed.dims, seed=0)
    F = (2e-6, -1e-6, 1e-5)
    lat = SparseLattice(torch.from_numpy(bed.flags).cuda(), "lex", (8, 8, 8), bed.periodic)
    cells = lat.cells().cpu().numpy()
    n = lat.n
    alpha = torch.from_numpy(alpha_dense.reshape(-1)[cells].copy()).cuda()
    c, w, _ = oracle.velocity_set()
    rng = np.random.default_rng(40 + K)
    f0 = torch.from_numpy(w[:, None] * (1.0 + 1e-3 * rng.standard_normal((19, n)))).cuda()
    # a direction with net axial momentum, so that <dJ/df0, v> is O(1)
    v = torch.from_numpy(w[:, None] * (np.asarray(c, np.float64)[:, 2:3]
                                       + 0.5 * rng.standard_normal((19, n)))).cuda()
    st = LBMState(lat, precision)
    st.set_damping(alpha)

    def J(f, Fv):
        st.set_pdfs(f)
        st.step(K, WP, WM, Fv)
        return st.reduce_flux(2)[1]

    def exact(fun, h):
        def central(e):
            return (fun(e) - fun(-e)) / (2 * e)
        return central(h) if K == 2 else (4 * central(h) - central(2 * h)) / 3

    st.set_pdfs(f0)
    adj = Adjoint(st, K)
    J0 = adj.forward(WP, WM, F, 2)
    dF, _, df0 = adj.backward(want_alpha=False, want_f0=True)
    assert abs(J0 - J(f0, F)) <= 1e-12 * abs(J0)
    d = exact(lambda e: J(f0 + e * v, F), 2e-3)
    dot = float((df0 * v).sum())
    err_f0 = abs(dot - d) / abs(d)
    dFx = []
    for k in range(3):
        def jf(e, k=k):
            Fe = list(F)
            Fe[k] += e
            return J(f0, tuple(Fe))
        dFx.append(exact(jf, 1e-5))
    # dJ/dF relative to its norm: J is the mean u_z, so the x and y
    # components are small cross terms
    err_F = _norm_rel(dF, dFx)
    print(f"{precision} K={K}: <dJ/df0, v> rel err {err_f0:.2e}; dJ/dF norm-rel err {err_F:.2e}")
    assert err_f0 <= tol and err_F <= tol, (err_f0, err_F)
    adj.close()
    st.close()
    lat.close()
