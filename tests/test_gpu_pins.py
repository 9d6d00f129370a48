"""GPU checks of properties the paper fixes independently of any implementation.

- Order within a colour class (Algorithm 1 with nine colours): boxes of one colour
  are at distance >= 3, so they touch disjoint blocks and the factorization does not
  depend on the order in which they are taken: a permuted order gives the same bits.
- Accuracy follows the tolerance (Tables "laplace2"): the relative residual of the
  direct solve stays below 10 eps and falls with eps.
- The factorization inverts the matrix it compresses (Eq. 9): solving A x, with A x
  formed exactly by FFT, returns x to about eps.
- Device memory handed back with rss_trim_memory does not change later results.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle.dense import relres
from oracle.rss import KernelSpec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15458_gb300 as P
    return P


def _solve(P, f, b):
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T if b.ndim == 2 else torch.from_numpy(b.copy()).cuda()
    P.rss_solve(f, bt)
    torch.cuda.synchronize()
    return bt.cpu().numpy()


@pytest.mark.parametrize("kind,kappa", [(0, 0.0), (1, 25.0)], ids=["laplace", "helmholtz"])
def test_order_within_a_colour_class_does_not_matter(P, kind, kappa):
    side = 128
    tree = P.rss_build_tree(W.grid_points(side), 64)
    f0 = P.rss_factor(tree, kind=kind, eps=1e-6, h=1 / side, kappa=kappa)
    f1 = P.rss_factor(tree, kind=kind, eps=1e-6, h=1 / side, kappa=kappa, class_order=12345)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(f0, g), P.rss_level_ranks(f1, g))
    for g, box in ((16, 0), (16, 137), (16, 255), (8, 27), (4, 5)):
        a, b = P.rss_box_record(f0, g, box), P.rss_box_record(f1, g, box)
        for key in ("S", "R", "C", "T", "LU", "piv", "E", "F"):
            assert np.array_equal(a[key], b[key]), (g, box, key)
    rhs = W.gaussian_rhs(side * side, 2, kind == 1, 31)
    assert np.array_equal(_solve(P, f0, rhs), _solve(P, f1, rhs))


def test_residual_follows_the_tolerance(P):
    side = 64
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    tree = P.rss_build_tree(pts, 64)
    b = W.gaussian_rhs(side * side, 1, False, 1000)
    res = []
    for eps in (1e-6, 1e-9, 1e-12):
        f = P.rss_factor(tree, kind=0, eps=eps, h=1 / side)
        r = relres(pts, spec, _solve(P, f, b), b)
        assert r <= 10 * eps, (eps, r)
        res.append(r)
    assert res[0] > res[1] > res[2]


@pytest.mark.parametrize("kind,kappa", [(0, 0.0), (1, 25.0)], ids=["laplace", "helmholtz"])
def test_solve_inverts_the_fft_matvec(P, kind, kappa):
    side, eps = 128, 1e-8
    tree = P.rss_build_tree(W.grid_points(side), 64)
    f = P.rss_factor(tree, kind=kind, eps=eps, h=1 / side, kappa=kappa)
    x = W.gaussian_rhs(side * side, 3, kind == 1, 77)
    xt = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().T
    b = P.rss_matvec(f, xt)
    P.rss_solve(f, b)
    torch.cuda.synchronize()
    y = b.cpu().numpy()
    assert np.linalg.norm(y - x) <= 10 * eps * np.linalg.norm(x)


def test_trimmed_pool_gives_the_same_factorization(P):
    side = 128
    tree = P.rss_build_tree(W.grid_points(side), 64)
    b = W.gaussian_rhs(side * side, 40, False, 9)
    f = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side)
    x0 = _solve(P, f, b)
    P.rss_free(f)
    P.rss_trim_memory(0)
    f = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side)
    assert np.array_equal(_solve(P, f, b), x0)
    P.rss_trim_memory(1 << 30)
