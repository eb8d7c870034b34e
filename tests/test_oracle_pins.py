"""Pins of the CPU oracle against closed forms, textbook identities and
brute force -- nothing here compares the oracle with itself.

Each pin is chosen so that a plausible slip in the oracle (a wrong
weight, a swapped velocity, a dropped forcing term, a misplaced wall, a
wrong key bit) fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1111_1129_gb300 import inputs

OMEGA_P = 1.0 / 0.8
OMEGA_M = oracle.omega_minus(OMEGA_P)          # Lambda = 3/16
NU = (1.0 / OMEGA_P - 0.5) / 3.0               # lattice viscosity, 0.1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_cells(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


# ---------------------------------------------------------------------------
# D3Q19 velocity set (Sec. 1): lattice isotropy up to fourth order.

def test_velocity_set_isotropy():
    c, w, opp = oracle.velocity_set()
    c = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(c[opp], -c)
    assert sorted(map(tuple, c.astype(int).tolist())) == sorted(
        [(0, 0, 0)] + [v for v in itertools.product((-1, 0, 1), repeat=3)
                       if sum(abs(x) for x in v) in (1, 2)])
    np.testing.assert_allclose(np.einsum("q,qa->a", w, c), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), iso4, atol=1e-16)


# ---------------------------------------------------------------------------
# One collision: conservation and the equilibrium's moments.

def _random_g(rng, scale=1e-2):
    _, w, _ = oracle.velocity_set()
    return w * (1.0 + scale * rng.standard_normal(19))


@pytest.mark.parametrize("alpha", [0.0, 0.037])
def test_collision_conserves_mass_and_balances_momentum(alpha):
    c, _, _ = oracle.velocity_set()
    rng = np.random.default_rng(1)
    for _ in range(20):
        g = _random_g(rng)
        F = 1e-3 * rng.standard_normal(3)
        fo, rho, u = oracle.collide(g, F, alpha, OMEGA_P, OMEGA_M)
        assert abs(rho - g.sum()) < 1e-15
        assert abs((fo - g).sum()) < 1e-15 * rho
        j = c.T.astype(float) @ g
        np.testing.assert_allclose(u, (j + 0.5 * F) / (1.0 + 0.5 * alpha), rtol=0, atol=1e-17)
        # the collision adds exactly the damped body force to the momentum
        # (rounding of 19 differences of O(0.05) values: ~1e-16)
        np.testing.assert_allclose(c.T.astype(float) @ (fo - g), F - alpha * u, rtol=0,
                                   atol=2e-16)


def test_equilibrium_moments_via_bgk_unit_relaxation():
    """With omega+ = omega- = 1 and no force, f* is the equilibrium itself,
    whose D3Q19 moments are rho, u and rho/3 I + u u (incompressible form,
    rho0 = 1)."""
    c, _, _ = oracle.velocity_set()
    c = c.astype(float)
    rng = np.random.default_rng(2)
    for _ in range(10):
        g = _random_g(rng, 5e-2)
        e, rho, u = oracle.collide(g, np.zeros(3), 0.0, 1.0, 1.0)
        assert abs(e.sum() - rho) < 1e-15
        np.testing.assert_allclose(c.T @ e, u, atol=1e-17)
        np.testing.assert_allclose(np.einsum("q,qa,qb->ab", e, c, c),
                                   rho / 3.0 * np.eye(3) + np.outer(u, u), atol=1e-16)


# ---------------------------------------------------------------------------
# Streaming (pull, Sec. 7) and implicit bounce back (Sec. 2) in isolation:
# omega+ = omega- = 0 and F = 0 turn the collision into the identity.

def test_pure_streaming_is_a_roll_on_a_periodic_box():
    rng = np.random.default_rng(3)
    flags = np.zeros((5, 4, 3), np.uint8)
    c, _, _ = oracle.velocity_set()
    f0 = rng.random((19,) + flags.shape)
    t = 4
    f, _, _, _ = oracle.run(flags, 7, 0.0, 0.0, np.zeros(3), t, f=f0)
    for q in range(19):
        ref = np.roll(f0[q], shift=(t * c[q, 2], t * c[q, 1], t * c[q, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(f[q], ref)


def test_pure_streaming_bounce_back_cycle_in_a_closed_box():
    """A PDF travelling along x in a closed 5-cell box bounces at both faces
    and is back where it started after 2*5 steps."""
    rng = np.random.default_rng(4)
    flags = np.zeros((1, 1, 5), np.uint8)
    f0 = rng.random((19,) + flags.shape)
    f, _, _, _ = oracle.run(flags, 0b110, 0.0, 0.0, np.zeros(3), 10, f=f0)
    np.testing.assert_array_equal(f, f0)
    f, _, _, _ = oracle.run(flags, 0b110, 0.0, 0.0, np.zeros(3), 5, f=f0)
    assert not np.array_equal(f, f0)


def test_pure_streaming_permutes_slots_with_solids():
    rng = np.random.default_rng(5)
    flags = (rng.random((6, 5, 7)) < 0.3).astype(np.uint8)
    f0 = rng.random((19,) + flags.shape)
    f, _, _, _ = oracle.run(flags, 0b100, 0.0, 0.0, np.zeros(3), 3, f=f0)
    fl = flags == 0
    np.testing.assert_array_equal(np.sort(f[:, fl].ravel()), np.sort(f0[:, fl].ravel()))


# ---------------------------------------------------------------------------
# Whole-solver closed forms.

def test_uniform_acceleration_in_a_periodic_box():
    """All-fluid periodic box: every cell sees the same state; step t sees
    momentum j_t with u_t = (j_t + F/2)/(1 + alpha/2) and the collision adds
    F - alpha u_t.  For alpha = 0 that is u_t = (t - 1/2) F."""
    flags = np.zeros((5, 4, 3), np.uint8)
    F = np.array([1e-3, -2e-3, 5e-4])
    n = flags.size
    for alpha in (0.0, 0.02):
        a = np.full(flags.shape, alpha)
        steps = 7
        _, obs, rho, u = oracle.run(flags, 7, OMEGA_P, OMEGA_M, F, steps, alpha=a)
        j = np.zeros(3)
        for t in range(steps):
            ut = (j + 0.5 * F) / (1.0 + 0.5 * alpha)
            np.testing.assert_allclose(obs[t, 1:] / n, ut, rtol=1e-12, atol=1e-18)
            assert abs(obs[t, 0] - n) < 1e-12 * n
            j = j + F - alpha * ut
        np.testing.assert_allclose(u[:, 0, 0, 0], ut, rtol=1e-12)
        if alpha == 0.0:
            np.testing.assert_allclose(ut, (steps - 0.5) * F, rtol=1e-12)
        np.testing.assert_allclose(rho, 1.0, rtol=1e-14)


def _poiseuille(H):
    y = np.arange(H) + 0.5
    return y * (H - y)


@pytest.mark.parametrize("walls", ["faces", "solid_rows"])
def test_plane_poiseuille_exact_at_magic_lambda(walls):
    """TRT with Lambda = 3/16 and half-way bounce back reproduces the
    parabolic profile u(y) = F/(2 nu) y (H - y), walls at y = 0 and y = H,
    to round-off."""
    H, Fz = 8, 1e-5
    if walls == "faces":
        flags = np.zeros((1, H, 1), np.uint8)
        periodic = 0b101
    else:
        flags = np.zeros((1, H + 2, 1), np.uint8)
        flags[:, 0, :] = 1
        flags[:, -1, :] = 1
        periodic = 0b111
    _, _, _, u = oracle.run(flags, periodic, OMEGA_P, OMEGA_M, [0.0, 0.0, Fz], 4000)
    uz = u[2, 0, :, 0] if walls == "faces" else u[2, 0, 1:-1, 0]
    ref = Fz / (2 * NU) * _poiseuille(H)
    assert np.max(np.abs(uz - ref)) / np.max(ref) < 1e-10
    # no cross flow beyond the round-off of j = sum c g over O(0.05) PDFs
    assert np.max(np.abs(u[0])) < 1e-11 * np.max(ref)
    assert np.max(np.abs(u[1])) < 1e-11 * np.max(ref)


def test_plane_poiseuille_not_exact_off_magic_lambda():
    H, Fz = 8, 1e-5
    flags = np.zeros((1, H, 1), np.uint8)
    om = oracle.omega_minus(OMEGA_P, 0.25)
    _, _, _, u = oracle.run(flags, 0b101, OMEGA_P, om, [0.0, 0.0, Fz], 4000)
    ref = Fz / (2 * NU) * _poiseuille(H)
    assert np.max(np.abs(u[2, 0, :, 0] - ref)) / np.max(ref) > 1e-4


def _duct(H, F, nu, nterms=401):
    """Fourier-series solution of nu Lap u = -F in a square of side H with
    no-slip walls, at the cell centres."""
    a = H / 2.0
    Y = np.arange(H) + 0.5 - a
    yy, zz = np.meshgrid(Y, Y, indexing="ij")
    u = np.zeros_like(yy)
    for i in range(1, nterms + 1, 2):
        k = i * math.pi / (2 * a)
        ratio = np.exp(k * (np.abs(zz) - a)) * (1 + np.exp(-2 * k * np.abs(zz))) / (
            1 + np.exp(-2 * k * a))
        u += (-1) ** ((i - 1) // 2) * (1 - ratio) * np.cos(k * yy) / i ** 3
    return 16 * a * a * F / (nu * math.pi ** 3) * u


def test_square_duct_second_order_convergence():
    errs = []
    for H in (6, 12):
        flags = np.zeros((H, H, 1), np.uint8)
        _, _, _, u = oracle.run(flags, 0b001, OMEGA_P, OMEGA_M, [1e-5, 0.0, 0.0], 3000)
        ux = u[0, :, :, 0].T          # [y, z]
        ref = _duct(H, 1e-5, NU)
        errs.append(np.linalg.norm(ux - ref) / np.linalg.norm(ref))
    assert errs[1] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.5


def test_mirror_and_axis_swap_symmetry():
    rng = np.random.default_rng(6)
    flags = (rng.random((8, 6, 6)) < 0.25).astype(np.uint8)
    F = [0.0, 0.0, 1e-4]
    steps = 6
    _, _, _, u = oracle.run(flags, 0b100, OMEGA_P, OMEGA_M, F, steps)
    scale = np.abs(u).max()
    # mirror y -> Ny-1-y: u_y flips sign
    _, _, _, um = oracle.run(flags[:, ::-1, :].copy(), 0b100, OMEGA_P, OMEGA_M, F, steps)
    np.testing.assert_allclose(um[0], u[0][:, ::-1, :], atol=1e-13 * scale)
    np.testing.assert_allclose(um[1], -u[1][:, ::-1, :], atol=1e-13 * scale)
    np.testing.assert_allclose(um[2], u[2][:, ::-1, :], atol=1e-13 * scale)
    # swap x and y: flags'[z, y', x'] = flags[z, x', y']
    _, _, _, us = oracle.run(flags.transpose(0, 2, 1).copy(), 0b100, OMEGA_P, OMEGA_M, F, steps)
    np.testing.assert_allclose(us[0], u[1].transpose(0, 2, 1), atol=1e-13 * scale)
    np.testing.assert_allclose(us[1], u[0].transpose(0, 2, 1), atol=1e-13 * scale)
    np.testing.assert_allclose(us[2], u[2].transpose(0, 2, 1), atol=1e-13 * scale)


def test_mass_is_conserved_over_a_run():
    bed = inputs.bed_small()
    _, obs, _, _ = oracle.run(bed.flags, bed.periodic, OMEGA_P, OMEGA_M, [0, 0, 1e-6], 50)
    n = bed.n_fluid
    np.testing.assert_allclose(obs[:, 0], n, rtol=1e-13)
    assert np.all(np.diff(obs[:, 3]) > 0)       # accelerating from rest


# ---------------------------------------------------------------------------
# The sparse representation (Sec. 2-3).

def _order_cells(cells, dims):
    nx, ny, _ = dims
    return [(int(c % nx), int((c // nx) % ny), int(c // (nx * ny))) for c in cells]


def test_lex_order_and_contiguous_index():
    rng = np.random.default_rng(7)
    flags = (rng.random((5, 6, 7)) < 0.4).astype(np.uint8)
    cells, inv, adj = oracle.build_sparse(flags, oracle.ORDER_LEX)
    np.testing.assert_array_equal(cells, np.flatnonzero(flags.ravel() == 0))
    assert len(cells) == int((flags == 0).sum())
    np.testing.assert_array_equal(inv.ravel()[cells], np.arange(len(cells)))
    assert np.all(inv[flags == 1] == -1)


def test_blocked_order_golden_and_invariants():
    dims = (5, 3, 2)
    flags = np.zeros(dims[::-1], np.uint8)
    cells, _, _ = oracle.build_sparse(flags, oracle.ORDER_BLOCKED, (2, 2, 2))
    assert _order_cells(cells, dims) == _golden_cells("blocked2_5x3x2_order.txt")
    rng = np.random.default_rng(8)
    flags = (rng.random((6, 5, 7)) < 0.3).astype(np.uint8)
    lex, _, ladj = oracle.build_sparse(flags, oracle.ORDER_LEX, periodic=5)
    for b in [(1, 1, 1), (7, 7, 7), (100, 100, 100)]:
        blk, _, badj = oracle.build_sparse(flags, oracle.ORDER_BLOCKED, b, periodic=5)
        np.testing.assert_array_equal(blk, lex)
        np.testing.assert_array_equal(badj, ladj)


def _morton_recursive(size, fanout):
    """Cells of a size^3 cube in Z-curve order by octant recursion: at every
    level split into fanout^3 sub-cubes, visited lexicographically."""
    out = []

    def rec(x0, y0, z0, s):
        if s == 1:
            out.append((x0, y0, z0))
            return
        h = s // fanout
        for dz in range(fanout):
            for dy in range(fanout):
                for dx in range(fanout):
                    rec(x0 + dx * h, y0 + dy * h, z0 + dz * h, h)

    rec(0, 0, 0, size)
    return out


def test_morton_orders_match_octant_recursion():
    flags = np.zeros((8, 8, 8), np.uint8)
    cells, _, _ = oracle.build_sparse(flags, oracle.ORDER_MORTON1)
    assert _order_cells(cells, (8, 8, 8)) == _morton_recursive(8, 2)
    flags16 = np.zeros((16, 16, 16), np.uint8)
    cells, _, _ = oracle.build_sparse(flags16, oracle.ORDER_MORTON2)
    assert _order_cells(cells, (16, 16, 16)) == _morton_recursive(16, 4)
    flags4 = np.zeros((4, 4, 4), np.uint8)
    cells, _, _ = oracle.build_sparse(flags4, oracle.ORDER_MORTON1)
    assert _order_cells(cells, (4, 4, 4))[:16] == _golden_cells("morton1_4x4x4_first16.txt")


def test_morton_non_power_of_two_is_the_cube_order_restricted():
    """On a box that is not a power-of-two cube the order is the Z curve of
    the enclosing cube with cells outside the box skipped."""
    dims = (6, 3, 5)
    flags = np.zeros(dims[::-1], np.uint8)
    cells, _, _ = oracle.build_sparse(flags, oracle.ORDER_MORTON1)
    ref = [p for p in _morton_recursive(8, 2) if p[0] < 6 and p[1] < 3 and p[2] < 5]
    assert _order_cells(cells, dims) == ref


@pytest.mark.parametrize("kind,block", [(0, (1, 1, 1)), (1, (2, 3, 2)), (2, (1, 1, 1)),
                                        (3, (1, 1, 1))])
@pytest.mark.parametrize("periodic", [0, 0b010, 0b111])
def test_adjacency_is_a_permutation_and_matches_dense_streaming(kind, block, periodic):
    rng = np.random.default_rng(9 + kind + periodic)
    flags = (rng.random((5, 6, 4)) < 0.35).astype(np.uint8)
    cells, _, adj = oracle.build_sparse(flags, kind, block, periodic)
    n = len(cells)
    slots = np.concatenate([np.arange(n), adj.ravel()])
    np.testing.assert_array_equal(np.sort(slots), np.arange(19 * n))
    # pure streaming on the dense grid == one gather through the adjacency
    f0 = rng.random((19,) + flags.shape)
    f1, _, _, _ = oracle.run(flags, periodic, 0.0, 0.0, np.zeros(3), 1, f=f0)
    sp0 = oracle.to_sparse(f0, cells).ravel()
    sp1 = np.concatenate([sp0[:n], sp0[adj.ravel()]])
    np.testing.assert_array_equal(sp1, oracle.to_sparse(f1, cells).ravel())


def test_keys_are_injective():
    for kind, block in [(0, (1, 1, 1)), (1, (3, 2, 4)), (2, (1, 1, 1)), (3, (1, 1, 1))]:
        k = oracle.keys(kind, (7, 5, 6), block)
        assert len(np.unique(k)) == k.size


# ---------------------------------------------------------------------------
# Adjoint against central finite differences of the forward oracle.

def _adjoint_case():
    rng = np.random.default_rng(10)
    flags = (rng.random((6, 4, 5)) < 0.25).astype(np.uint8)
    alpha = 0.05 * rng.random(flags.shape)
    F = np.array([1e-4, 2e-4, 1e-3])
    _, w, _ = oracle.velocity_set()
    f0 = oracle.rest_state(flags) * (1.0 + 0.01 * rng.standard_normal((19,) + flags.shape))
    return rng, flags, alpha, F, f0


def _J(flags, F, alpha, f0, steps, axis=2):
    _, obs, _, _ = oracle.run(flags, 0b100, OMEGA_P, OMEGA_M, F, steps, alpha=alpha, f=f0)
    return obs[-1, 1 + axis] / int((flags == 0).sum())


def test_adjoint_matches_finite_differences():
    rng, flags, alpha, F, f0 = _adjoint_case()
    K = 6
    J, dF, da, lam0 = oracle.adjoint(flags, 0b100, OMEGA_P, OMEGA_M, F, K, 2, alpha=alpha, f0=f0)
    assert abs(J - _J(flags, F, alpha, f0, K)) < 1e-15
    for k in range(3):
        h = 1e-6
        Fp, Fm = F.copy(), F.copy()
        Fp[k] += h
        Fm[k] -= h
        fd = (_J(flags, Fp, alpha, f0, K) - _J(flags, Fm, alpha, f0, K)) / (2 * h)
        assert abs(dF[k] - fd) < 1e-7 * max(abs(fd), 1e-3), (k, dF[k], fd)
    fluid = np.argwhere(flags == 0)
    for idx in fluid[rng.choice(len(fluid), 4, replace=False)]:
        idx = tuple(idx)
        h = 1e-5
        ap, am = alpha.copy(), alpha.copy()
        ap[idx] += h
        am[idx] -= h
        fd = (_J(flags, F, ap, f0, K) - _J(flags, F, am, f0, K)) / (2 * h)
        assert abs(da[idx] - fd) < 1e-6 * abs(fd) + 1e-13, (idx, da[idx], fd)
    assert np.all(da[flags == 1] == 0.0)
    # directional derivative with respect to the initial state
    v = rng.standard_normal(f0.shape) * (flags == 0)
    h = 1e-6
    fd = (_J(flags, F, alpha, f0 + h * v, K) - _J(flags, F, alpha, f0 - h * v, K)) / (2 * h)
    assert abs(np.sum(lam0 * v) - fd) < 1e-7 * abs(fd)


@pytest.mark.parametrize("K", [2, 3])
def test_adjoint_equals_exact_directional_derivatives(K):
    """The dot-product test of the transposed Jacobian, to round-off.  One
    step is a quadratic polynomial of the state and of F (u is linear in
    the pulled values and in F; the equilibrium is quadratic in u; rho0 = 1
    divides nothing), and J is linear in the last pulled values.  So J after
    K = 2 steps is a polynomial of degree 2 in f0 along any direction v, and
    in F: its central difference is the exact derivative whatever h.  After
    K = 3 steps it has degree 4, and (4 D(h) - D(2h)) / 3 cancels the h^2
    term of the central difference D.  <dJ/df0, v> and dJ/dF must match
    these to round-off (a wrong sign, index or transposition in the reverse
    step would show at O(1))."""
    rng, flags, alpha, F, f0 = _adjoint_case()
    J, dF, _, lam0 = oracle.adjoint(flags, 0b100, OMEGA_P, OMEGA_M, F, K, 2, alpha=alpha, f0=f0)

    def exact(fun, h):
        def central(e):
            return (fun(e) - fun(-e)) / (2 * e)
        return central(h) if K == 2 else (4 * central(h) - central(2 * h)) / 3

    v = rng.standard_normal(f0.shape) * (flags == 0)
    d = exact(lambda e: _J(flags, F, alpha, f0 + e * v, K), 1e-2)
    assert abs(np.sum(lam0 * v) - d) <= 1e-12 * abs(d), (np.sum(lam0 * v), d)
    for k in range(3):
        def jf(e, k=k):
            Fe = F.copy()
            Fe[k] += e
            return _J(flags, Fe, alpha, f0, K)
        d = exact(jf, 1e-3)
        assert abs(dF[k] - d) <= 1e-12 * abs(d), (k, dF[k], d)


# ---------------------------------------------------------------------------
# Hilbert curve (named among the numbering schemes in Sec. 3).

@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_hilbert_is_continuous_and_recursive(n):
    """On a 2^k cube the Hilbert order starts at the origin, steps to a face
    neighbour every time, and visits every aligned run of 8^j cells as one
    2^j sub-cube (its recursive construction)."""
    flags = np.zeros((n, n, n), np.uint8)
    cells, _, _ = oracle.build_sparse(flags, oracle.ORDER_HILBERT)
    xyz = np.stack([cells % n, (cells // n) % n, cells // (n * n)], axis=1)
    assert tuple(xyz[0]) == (0, 0, 0)
    assert np.all(np.abs(np.diff(xyz, axis=0)).sum(axis=1) == 1)
    j = 1
    while 2 ** j <= n:
        run = 8 ** j
        for b in range(0, n ** 3, run):
            block = xyz[b:b + run]
            assert np.all(block.max(axis=0) - block.min(axis=0) == 2 ** j - 1)
            assert np.all(block.min(axis=0) % 2 ** j == 0)
        j += 1


def test_hilbert_non_power_of_two_is_the_cube_order_restricted():
    dims = (6, 3, 5)
    flags = np.zeros(dims[::-1], np.uint8)
    cells, _, _ = oracle.build_sparse(flags, oracle.ORDER_HILBERT)
    cube = np.zeros((8, 8, 8), np.uint8)
    cc, _, _ = oracle.build_sparse(cube, oracle.ORDER_HILBERT)
    ref = [(int(c % 8), int((c // 8) % 8), int(c // 64)) for c in cc]
    ref = [p for p in ref if p[0] < 6 and p[1] < 3 and p[2] < 5]
    assert _order_cells(cells, dims) == ref
