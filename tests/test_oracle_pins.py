"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to the mathematics, a textbook table, a
library special case, or an exactness property, so that a dropped term, a
wrong sign, a missing conjugate or a transposed operand fails at least one.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy import special

import workloads as W
from oracle import rss
from oracle.dense import dense_matrix, fft_matvec, relres
from oracle.rss import KernelSpec, cpqr_id, factor, solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------- kernels
def test_helmholtz_kernel_matches_bessel_table():
    """(i/4) H0^(1)(kappa r) (Eq. 18) against Abramowitz & Stegun Table 9.1."""
    rows = np.loadtxt(os.path.join(GOLDEN, "bessel_j0_y0.txt"))
    spec = KernelSpec("helmholtz", h=1.0, kappa=1.0)
    for x, j0, y0 in rows:
        k = rss.kernel_block(spec, np.array([[x, 0.0]]), np.zeros((1, 2)))[0, 0]
        assert abs(k.real - (-y0 / 4)) < 1e-14
        assert abs(k.imag - (j0 / 4)) < 1e-14


def test_kernels_solve_their_pdes():
    """Laplace kernel is harmonic, Helmholtz kernel solves (Delta + kappa^2) K = 0 off the origin."""
    d = 1e-3
    x0 = np.array([0.37, -0.21])
    st = np.array([[0, 0], [d, 0], [-d, 0], [0, d], [0, -d]]) + x0
    for spec, k2 in ((KernelSpec("laplace", h=1.0), 0.0),
                     (KernelSpec("helmholtz", h=1.0, kappa=7.0), 49.0)):
        v = rss.kernel_block(spec, st, np.zeros((1, 2)))[:, 0]
        lap = (v[1] + v[2] + v[3] + v[4] - 4 * v[0]) / d ** 2
        assert abs(lap + k2 * v[0]) < 1e-5 * max(1.0, abs(k2 * v[0]))
    # Laplace: K(r) - K(2r) = (1 / 2 pi) log 2 with h = 1
    spec = KernelSpec("laplace", h=1.0)
    k = rss.kernel_block(spec, np.array([[0.3, 0.4], [0.6, 0.8]]), np.zeros((1, 2)))[:, 0]
    assert abs((k[0] - k[1]) - np.log(2) / (2 * np.pi)) < 1e-15


def test_entries_diagonal_rule():
    pts = W.grid_points(4)
    idx = np.arange(16)
    A = rss.entries(KernelSpec("laplace", h=0.25, diag=1.0), pts, idx, idx)
    assert np.all(np.diag(A) == 1.0)
    assert np.allclose(A, A.T)


# --------------------------------------------------------------------------- ID
@pytest.mark.parametrize("seed", range(4))
def test_cpqr_pivots_match_lapack_geqp3(seed):
    """Full-rank CPQR (eps = 0) picks the same pivots as LAPACK geqp3 and the same |R|."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((40, 12)) * rng.uniform(0.1, 3.0, 12)
    k, perm, T, R = cpqr_id(Y, 0.0)
    Rs, piv = sla.qr(Y, mode="r", pivoting=True)
    assert k == 12
    assert np.array_equal(perm, piv)
    assert np.allclose(np.abs(np.diag(R[:12])), np.abs(np.diag(Rs)), rtol=1e-12)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("eps", [1e-2, 1e-5, 1e-9])
def test_cpqr_is_an_id_and_truncates_first(cplx, eps):
    """Definition 1: ||Y_R - Y_S T||_F <= eps ||Y||_F, and k is the first rank that meets it."""
    rng = np.random.default_rng(7)
    m, n = 60, 24
    # numerically low-rank matrix with geometrically decaying singular values
    U, _ = np.linalg.qr(rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0))
    Y = (U * (0.3 ** np.arange(n))) @ V.conj().T
    k, perm, T, R = cpqr_id(Y, eps)
    S, Rr = perm[:k], perm[k:]
    res = np.linalg.norm(Y[:, Rr] - Y[:, S] @ T)
    assert res <= eps * np.linalg.norm(Y) * (1 + 1e-8)
    assert abs(res - np.linalg.norm(R[k:, k:])) <= 1e-12 * np.linalg.norm(Y) + 1e-6 * res
    if k > 0:   # with one skeleton column fewer (same pivot order) the bound fails
        S1, R1 = perm[:k - 1], perm[k - 1:]
        T1 = np.linalg.lstsq(Y[:, S1], Y[:, R1], rcond=None)[0] if k > 1 else np.zeros((0, n - k + 1))
        assert np.linalg.norm(Y[:, R1] - Y[:, S1] @ T1) > eps * np.linalg.norm(Y)


def test_cpqr_exact_low_rank_and_ties():
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((50, 5)) @ rng.standard_normal((5, 20))
    k, perm, T, _ = cpqr_id(Y, 1e-12)
    assert k == 5
    assert np.linalg.norm(Y[:, perm[k:]] - Y[:, perm[:k]] @ T) < 1e-12 * np.linalg.norm(Y)
    # duplicated columns tie exactly: the lowest original column must win
    Z = np.hstack([Y[:, :3], Y[:, :3]])
    k, perm, _, _ = cpqr_id(Z, 0.0)
    assert perm[0] < 3


def _orthogonal_columns(norms2, scale=1.0):
    """Columns that are scaled, distinct unit vectors: a Householder step mixes only
    the rows of the pivot, so every downdated norm stays exact and the pivot choice
    depends on the given squared norms alone."""
    n = len(norms2)
    Y = np.zeros((n + 2, n))
    Y[np.arange(n), np.arange(n)] = np.sqrt(np.asarray(norms2, dtype=float)) * scale
    return Y


@pytest.mark.parametrize("scale", [1.0, 1e-5, 1e4])
def test_cpqr_tie_window(scale):
    """The pivot rule: the largest remaining squared norm wins unless another column
    lies within 1e-6 of it (relative), and among those the lowest original column
    wins.  A window of 1e-4 would take the lower column at 2e-6 apart; a window of
    1e-8 (or none) would take the larger one at 1e-7 apart.  The rule is relative,
    so scaling Y changes nothing."""
    for delta, first in ((2e-6, 1), (1e-7, 0), (5e-6, 1), (5e-7, 0)):
        _, perm, _, _ = cpqr_id(_orthogonal_columns([1.0, 1.0 + delta, 0.5, 0.25], scale), 0.0)
        assert perm[0] == first, (delta, perm)
    # the same window at a later step (column 0 is taken first, then 1 and 2 compete)
    for delta, second in ((2e-6, 2), (1e-7, 1)):
        _, perm, _, _ = cpqr_id(_orthogonal_columns([4.0, 1.0, 1.0 + delta, 0.25], scale), 0.0)
        assert perm[0] == 0 and perm[1] == second, (delta, perm)
    # a larger column that comes first in the original order wins either way
    _, perm, _, _ = cpqr_id(_orthogonal_columns([1.0 + 2e-6, 1.0, 0.5], scale), 0.0)
    assert perm[0] == 0


def test_cpqr_tie_window_absolute_floor():
    """Deep in the ID the remaining norms are tiny next to the largest initial one
    (y2max), and their rounding noise is set by y2max: columns within
    1e-12 sqrt(n_max y2max) of the maximum n_max count as tied as well."""
    # y2max = 1, n_max = 1e-13: the floor is 1e-12 * sqrt(1e-13) = 3.2e-19 (the
    # relative part adds 1e-19)
    _, perm, _, _ = cpqr_id(_orthogonal_columns([1.0, 1e-13, 1e-13 + 2e-19]), 0.0)
    assert list(perm[:2]) == [0, 1]
    _, perm, _, _ = cpqr_id(_orthogonal_columns([1.0, 1e-13, 1e-13 + 1e-18]), 0.0)
    assert list(perm[:2]) == [0, 2]


def test_cpqr_of_conjugate_stack_equals_real_stack():
    """[X; conj X] and [Re X; Im X] have proportional Gram matrices (2 Re X^H X),
    so column-pivoted QR gives both the same pivots and rank, and T is real."""
    rng = np.random.default_rng(11)
    U = rng.standard_normal((120, 12)) + 1j * rng.standard_normal((120, 12))
    V = rng.standard_normal((12, 40)) + 1j * rng.standard_normal((12, 40))
    X = (U * np.logspace(0, -11, 12)) @ V
    eps = 1e-7
    kc, pc, Tc, _ = cpqr_id(np.vstack([X, X.conj()]), eps)
    kr, pr, Tr, _ = cpqr_id(np.vstack([X.real, X.imag]), eps)
    assert kc == kr and 0 < kc < 40
    assert np.array_equal(pc, pr)
    # rounding in T grows with cond(R11), up to about 1/eps at the truncation
    tol = 1e-14 / eps
    assert np.abs(Tc.imag).max() <= tol * np.abs(Tc).max()
    assert np.abs(Tc.real - Tr).max() <= tol * np.abs(Tr).max()


def test_helmholtz_interpolation_matrices_stay_real():
    """A complex symmetric kernel keeps A complex symmetric through the
    eliminations (T real up to rounding), so every box's stack has the form
    [X; conj X]: the premise of computing the Helmholtz ID in real arithmetic."""
    side = 32
    fac = factor(W.grid_points(side), KernelSpec("helmholtz", h=1 / side, kappa=25.0), 1e-6, leaf=16)
    assert len(fac.records) > 0
    for rec in fac.records:
        if rec.T.size:
            assert np.abs(rec.T.imag).max() <= 1e-8 * max(1.0, np.abs(rec.T).max())


def test_cpqr_zero_matrix():
    k, perm, T, _ = cpqr_id(np.zeros((10, 4)), 1e-6)
    assert k == 0 and T.shape == (0, 4)


# --------------------------------------------------------------------------- LU and triangular solves
@pytest.mark.parametrize("seed", range(3))
def test_lu_matches_lapack_getrf(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((30, 30))
    LU, piv = rss.lu_factor_pp(A)
    LUs, pivs = sla.lu_factor(A)
    assert np.array_equal(piv, pivs)
    assert np.allclose(LU, LUs, rtol=1e-12, atol=1e-12)
    Ac = A + 1j * rng.standard_normal((30, 30))
    LU, piv = rss.lu_factor_pp(Ac)
    L = np.tril(LU, -1) + np.eye(30)
    assert np.allclose(rss.apply_row_swaps(piv, Ac), L @ np.triu(LU), atol=1e-12)
    b = rng.standard_normal((30, 3))
    assert np.allclose(rss.lu_solve_pp(LU, piv, b), np.linalg.solve(Ac, b), atol=1e-11)


def test_triangular_solves_match_scipy():
    rng = np.random.default_rng(11)
    U = np.triu(rng.standard_normal((9, 9))) + 4 * np.eye(9)
    B = rng.standard_normal((9, 5))
    assert np.allclose(rss.upper_solve(U, B), sla.solve_triangular(U, B), atol=1e-13)
    X = rng.standard_normal((7, 9))
    assert np.allclose(rss.right_upper_solve(X, U) @ U, X, atol=1e-12)
    L = np.tril(rng.standard_normal((9, 9)), -1)
    assert np.allclose(rss.unit_lower_solve(L, B),
                       sla.solve_triangular(L + np.eye(9), B, lower=True, unit_diagonal=True),
                       atol=1e-12)


# --------------------------------------------------------------------------- FFT matvec
@pytest.mark.parametrize("kind", ["laplace", "helmholtz", "rpoly"])
def test_fft_matvec_equals_dense(kind):
    side = 16
    pts, _ = W.shuffled(W.grid_points(side), 4)
    spec = KernelSpec(kind, h=1 / side, kappa=25.0, coef=(0.2, 0.5, -0.3), scale=0.1)
    # (the phase-weighted 'poly' kernel is not translation invariant, so no FFT)
    x = W.gaussian_rhs(side * side, 2, spec.is_complex, 9)
    assert np.allclose(fft_matvec(pts, spec, x), dense_matrix(pts, spec) @ x, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------- whole factorization
POLY = KernelSpec("poly", h=1 / 32, coef=(0.3, 0.5 - 0.2j, 0.7, 0.1 + 0.4j), scale=0.02, diag=1.0,
                  phase=(3.0, -2.0))
RPOLY = KernelSpec("rpoly", h=1 / 32, coef=(0.3, 0.5, -0.7, 0.4), scale=0.02, diag=1.0)


def _exact_case(spec, side=32, leaf=16, nrhs=2, seed=5):
    pts = W.grid_points(side)
    fac = factor(pts, spec, 1e-13, leaf=leaf)
    b = W.gaussian_rhs(side * side, nrhs, spec.is_complex, seed)
    A = dense_matrix(pts, spec)
    x = solve(fac, b)
    return fac, np.linalg.norm(A @ x - b) / np.linalg.norm(b)


@pytest.mark.parametrize("spec", [POLY, RPOLY], ids=["complex", "real"])
def test_rss_exact_when_far_field_is_exactly_low_rank(spec):
    """A polynomial kernel in z has an exactly low-rank far field that the proxy
    circle captures, so RS-S must reproduce A^{-1} b to rounding: this pins the
    sparsification, elimination, Schur updates, merge and both solve sweeps."""
    fac, rr = _exact_case(spec)
    assert rr < 1e-12
    assert min(fac.ranks[8]) < 16          # real compression took place
    assert len(fac.records) > 0


def test_rss_partitions_the_points():
    fac, _ = _exact_case(RPOLY)
    allR = np.concatenate([r.R for r in fac.records] + [fac.top_idx])
    assert np.array_equal(np.sort(allR), np.arange(32 * 32))


def test_rss_laplace_4096_against_dense_solve():
    """The 64 x 64 Laplace workload (eps = 1e-8): relres <= 10 eps and agreement with LU."""
    side = 64
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    fac = factor(pts, spec, 1e-8)
    b = W.gaussian_rhs(side * side, 1, False, 1000)
    x = solve(fac, b)
    A = dense_matrix(pts, spec)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * 1e-8
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * 1e-8
    assert abs(relres(pts, spec, x, b) - np.linalg.norm(A @ x - b) / np.linalg.norm(b)) < 1e-13


def test_rss_helmholtz_and_inverse_invariant():
    side = 32
    pts = W.grid_points(side)
    spec = KernelSpec("helmholtz", h=1 / side, kappa=25.0)
    fac = factor(pts, spec, 1e-6, leaf=16)
    xt = W.gaussian_rhs(side * side, 3, True, 77)
    b = fft_matvec(pts, spec, xt)
    x = solve(fac, b)
    assert relres(pts, spec, x, b) <= 10 * 1e-6
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= 10 * 1e-6


def test_rss_accuracy_follows_eps():
    """relres falls with eps (the pattern of Table 3)."""
    side = 32
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side, diag=0.05)
    b = W.gaussian_rhs(side * side, 1, False, 3)
    rr = [relres(pts, spec, solve(factor(pts, spec, e, leaf=16), b), b) for e in (1e-3, 1e-6, 1e-9)]
    assert rr[0] > rr[1] > rr[2]
    assert rr[1] < 1e-4 and rr[2] < 1e-7


def test_rss_user_order_does_not_matter():
    side = 32
    pts = W.grid_points(side)
    sp, p = W.shuffled(pts, 12)
    spec = KernelSpec("laplace", h=1 / side)
    b = W.gaussian_rhs(side * side, 1, False, 8)
    x1 = solve(factor(pts, spec, 1e-6, leaf=16), b)
    x2 = solve(factor(sp, spec, 1e-6, leaf=16), b[p])
    assert np.array_equal(x1[p], x2)


def test_proxy_id_reproduces_the_far_field():
    """Eq. (6): T from [A_MB; K_PB; A_BM^*; K_BP^*] also interpolates A_{F\\M,B} (Theorem 1)."""
    side = 64
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    grid = rss.grid_of(pts)
    g = 8
    lb = (grid.iy // 8) * g + (grid.ix // 8)
    local = (grid.iy % 8) * 8 + (grid.ix % 8)
    order = np.lexsort((local, lb))
    ptsl = list(np.split(order, np.cumsum(np.bincount(lb, minlength=g * g))[:-1]))
    blocks = {(b1, b2): rss.entries(spec, pts, ptsl[b1], ptsl[b2]) for b1 in range(g * g)
              for b2 in rss.stencil(b1, g)}
    B = 3 * g + 3
    L = 1.0 / g
    eps = 1e-7
    Y = rss.build_proxy_stack(spec, pts, blocks, ptsl, B, g, (3.5 * L, 3.5 * L), 1.25 * L, 64)
    k, perm, T, _ = cpqr_id(Y, eps)
    far = np.concatenate([ptsl[b] for b in range(g * g) if rss.chebyshev(b, B, g) > 2])
    AF = rss.entries(spec, pts, far, ptsl[B])
    err = np.linalg.norm(AF[:, perm[k:]] - AF[:, perm[:k]] @ T) / np.linalg.norm(AF)
    assert k < 64 and err < 100 * eps


# --------------------------------------------------------------------------- planted mistakes
def _planted(monkeypatch, name, fn):
    monkeypatch.setattr(rss, name, fn)
    return [_exact_case(POLY)[1], _exact_case(RPOLY)[1]]


def test_planted_mistake_dropped_term_is_caught(monkeypatch):
    orig = rss.sparsify

    def bad(A_SS, A_SR, A_RS, A_RR, A_NS, A_NR, A_SN, A_RN, T):
        X_CR, X_RC, X_RR = orig(A_SS, A_SR, A_RS, A_RR, A_NS, A_NR, A_SN, A_RN, T)
        return X_CR, X_RC, X_RR + T.conj().T @ (A_SR - A_SS @ T)   # drops -T^* X_SR
    assert max(_planted(monkeypatch, "sparsify", bad)) > 1e-8


def test_planted_mistake_missing_conjugate_is_caught(monkeypatch):
    orig = rss.sparsify

    def bad(A_SS, A_SR, A_RS, A_RR, A_NS, A_NR, A_SN, A_RN, T):
        return orig(A_SS, A_SR, A_RS, A_RR, A_NS, A_NR, A_SN, A_RN, T.conj())
    assert _planted(monkeypatch, "sparsify", bad)[0] > 1e-8


def test_planted_mistake_transposed_operand_is_caught(monkeypatch):
    orig = rss.eliminate

    def bad(X_CR, X_RC, X_RR):
        return orig(X_CR, X_RC, X_RR.T)
    assert max(_planted(monkeypatch, "eliminate", bad)) > 1e-8


def test_planted_mistake_wrong_sign_in_id_is_caught(monkeypatch):
    orig = rss.cpqr_id

    def bad(Y, eps):
        k, perm, T, R = orig(Y, eps)
        return k, perm, -T, R
    assert max(_planted(monkeypatch, "cpqr_id", bad)) > 1e-8


# --------------------------------------------------------------------------- paper discretisations (Section 5)
def test_self_integrals_match_adaptive_quadrature():
    """Eqs. 16 and 20: the closed-form / 1D reductions of the self-cell integral
    against scipy's 2D adaptive quadrature over the cell's four quadrants."""
    from scipy.integrate import dblquad
    for h in (1 / 32, 1 / 256):
        a = h / 2
        lap = 4 * dblquad(lambda y, x: -np.log(np.hypot(x, y)) / (2 * np.pi), 0, a, 0, a,
                          epsabs=1e-16, epsrel=1e-12)[0]
        assert abs(rss.self_integral("laplace", h) - lap) <= 1e-11 * abs(lap)
        for kappa in (25.0, 50.0):
            re = 4 * dblquad(lambda y, x: (0.25j * special.hankel1(0, kappa * np.hypot(x, y))).real,
                             0, a, 0, a, epsabs=1e-16, epsrel=1e-12)[0]
            im = 4 * dblquad(lambda y, x: (0.25j * special.hankel1(0, kappa * np.hypot(x, y))).imag,
                             0, a, 0, a, epsabs=1e-16, epsrel=1e-12)[0]
            v = rss.self_integral("helmholtz", h, kappa)
            assert abs(v - complex(re, im)) <= 1e-10 * abs(complex(re, im))


def test_lippmann_schwinger_matrix():
    """Eqs. 19-20: A = I + W (T + d I) W is complex symmetric, its diagonal is
    1 + kappa^2 b d, and the FFT matvec equals the dense one."""
    side = 16
    pts = W.grid_points(side)
    d = rss.self_integral("helmholtz", 1 / side, 25.0)
    spec = KernelSpec("ls", h=1 / side, kappa=25.0, diag=d)
    A = dense_matrix(pts, spec)
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
    b = np.exp(-32 * ((pts[:, 0] - 0.5) ** 2 + (pts[:, 1] - 0.5) ** 2))
    assert np.allclose(np.diag(A), 1 + 25.0 ** 2 * b * d, rtol=1e-14, atol=0)
    x = W.gaussian_rhs(side * side, 2, True, 3)
    assert np.abs(fft_matvec(pts, spec, x) - A @ x).max() <= 1e-12 * np.abs(A @ x).max()


def test_preconditioned_iterations_reach_1e12():
    """Section 5: PCG (Laplace, quadrature diagonal) and GMRES (Lippmann-Schwinger)
    with the RS-S factorization as preconditioner reach a relative residual of
    1e-12 in a few iterations; the result equals the dense solve."""
    from oracle.iterative import gmres, pcg
    side = 32
    pts = W.grid_points(side)
    h = 1 / side
    lap = KernelSpec("laplace", h=h, diag=rss.self_integral("laplace", h))
    fac = factor(pts, lap, 1e-6, leaf=16)
    b = W.gaussian_rhs(side * side, 1, False, 7)[:, 0]
    x, it, rel = pcg(lambda v: fft_matvec(pts, lap, v), lambda v: solve(fac, v), b)
    assert rel <= 1e-12 and 1 <= it <= 10
    A = dense_matrix(pts, lap)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
    ls = KernelSpec("ls", h=h, kappa=25.0, diag=rss.self_integral("helmholtz", h, 25.0))
    fac = factor(pts, ls, 1e-6, leaf=16)
    b = W.gaussian_rhs(side * side, 1, True, 8)[:, 0]
    x, it, rel = gmres(lambda v: fft_matvec(pts, ls, v), lambda v: solve(fac, v), b)
    assert rel <= 1e-12 and 1 <= it <= 10
    A = dense_matrix(pts, ls)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
