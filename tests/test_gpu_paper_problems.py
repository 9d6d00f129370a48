"""The paper's own discretisations on the GPU (Section 5), against the oracle.

* Laplace with the self-cell quadrature diagonal (Eq. 16), a first-kind
  system, refined by PCG with the RS-S factorization as preconditioner;
* the symmetrised Lippmann-Schwinger system (Eqs. 19-20, Gaussian bump),
  refined by GMRES(20).

The FFT matvec is compared with the oracle's FFT matvec, the factorization's
box records with the oracle's (same tolerances as the other parity tests),
and the iterative solutions with the dense solve; the final relative residual
is recomputed on the CPU by the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import rss as orss
from oracle.dense import dense_matrix, fft_matvec
from oracle.iterative import gmres, pcg
from oracle.rss import KernelSpec

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15458_gb300 as P
    return P


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def specs(side, kappa=25.0):
    h = 1 / side
    lap = KernelSpec("laplace", h=h, diag=orss.self_integral("laplace", h))
    ls = KernelSpec("ls", h=h, kappa=kappa, diag=orss.self_integral("helmholtz", h, kappa))
    return lap, ls


def factor_gpu(P, pts, spec, eps, leaf):
    tree = P.rss_build_tree(pts, leaf)
    kind = P.LAPLACE if spec.kind == "laplace" else P.HELMHOLTZ_LS
    return P.rss_factor(tree, kind=kind, eps=eps, h=spec.h, kappa=spec.kappa, diag_rule=1)


def test_self_integral_matches_oracle(P):
    for h in (1 / 64, 1 / 256, 1 / 2048):
        assert abs(P.rss_self_integral(P.LAPLACE, h) - orss.self_integral("laplace", h)) <= \
            1e-13 * abs(orss.self_integral("laplace", h))
        for kappa in (25.0, 50.0):
            o = orss.self_integral("helmholtz", h, kappa)
            assert abs(P.rss_self_integral(P.HELMHOLTZ_LS, h, kappa) - o) <= 1e-12 * abs(o)


@pytest.mark.parametrize("which", ["laplace", "ls"])
def test_fft_matvec_matches_oracle(P, which):
    side = 64
    pts, perm = W.shuffled(W.grid_points(side), 3)     # any user order
    spec = specs(side)[0 if which == "laplace" else 1]
    f = factor_gpu(P, pts, spec, 1e-6, 64)
    x = W.gaussian_rhs(side * side, 3, spec.is_complex, 9)
    xt = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().T
    y = P.rss_matvec(f, xt).cpu().numpy()
    ref = fft_matvec(pts, spec, x)
    assert rel(y, ref) <= 1e-12


def test_lippmann_schwinger_records_match_oracle(P):
    side, eps = 32, 1e-6
    pts = W.grid_points(side)
    spec = specs(side)[1]
    f = factor_gpu(P, pts, spec, eps, 16)
    fac = orss.factor(pts, spec, eps, leaf=16)
    for g in (8, 4):
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    tol = max(1e-10, 1e-14 / eps)
    for rec in fac.records:
        g = P.rss_box_record(f, rec.side, rec.box)
        assert np.array_equal(g["S"], rec.S) and np.array_equal(g["R"], rec.R)
        assert np.array_equal(g["C"], rec.C) and np.array_equal(g["piv"], rec.piv)
        for key, ref in (("T", rec.T), ("LU", rec.LU), ("E", rec.E), ("F", rec.F)):
            if ref.size:
                assert rel(g[key], ref) < tol, (rec.side, rec.box, key)
    b = W.gaussian_rhs(side * side, 1, True, 11)[:, 0]
    x = torch.from_numpy(b.copy()).cuda()
    P.rss_solve(f, x)
    assert rel(x.cpu().numpy(), orss.solve(fac, b)) < 1e-9


@pytest.mark.parametrize("which", ["laplace", "ls"])
def test_iterative_refinement_reaches_1e12(P, which):
    """PCG (Laplace, quadrature diagonal) / GMRES (Lippmann-Schwinger) with the GPU
    factorization as preconditioner: relres <= 1e-12 checked by the oracle's FFT
    matvec, x equal to the dense solve, iteration count equal to the oracle's."""
    side, eps = 64, 1e-6
    pts = W.grid_points(side)
    spec = specs(side)[0 if which == "laplace" else 1]
    f = factor_gpu(P, pts, spec, eps, 64)
    b = W.gaussian_rhs(side * side, 1, spec.is_complex, 21)[:, 0]
    x, it, relres = P.rss_solve_iterative(f, torch.from_numpy(b.copy()).cuda(), tol=1e-12)
    x = x.cpu().numpy()
    assert relres <= 1e-12 and 1 <= it <= 10
    assert np.linalg.norm(fft_matvec(pts, spec, x) - b) <= 2e-12 * np.linalg.norm(b)
    A = dense_matrix(pts, spec)
    assert rel(x, np.linalg.solve(A, b)) <= 1e-10
    fac = orss.factor(pts, spec, eps)
    solver = pcg if which == "laplace" else gmres
    _, it_o, _ = solver(lambda v: fft_matvec(pts, spec, v), lambda v: orss.solve(fac, v), b)
    assert abs(it - it_o) <= 1


def test_lippmann_schwinger_256_gmres(P):
    """The paper's Helmholtz problem at kappa = 25 on a 256 x 256 grid: GMRES(20)
    with the RS-S preconditioner (eps 1e-6) converges to 1e-12 in a few steps."""
    side = 256
    pts = W.grid_points(side)
    spec = specs(side)[1]
    f = factor_gpu(P, pts, spec, 1e-6, 64)
    b = W.gaussian_rhs(side * side, 1, True, 22)[:, 0]
    x, it, relres = P.rss_solve_iterative(f, torch.from_numpy(b.copy()).cuda(), tol=1e-12)
    assert relres <= 1e-12 and it <= 10
    assert np.linalg.norm(fft_matvec(pts, spec, x.cpu().numpy()) - b) <= 2e-12 * np.linalg.norm(b)
