"""Error statuses of rss_factor that come from the device: RSS_ENUMERIC (a zero
pivot in the LU of Eq. 8, which supposes X_RR non-singular) and RSS_ETIMEOUT (a
bounded barrier wait of the tensor-core Schur update that runs out).

Neither test faults or hangs the GPU.  The zero pivot is an exactly singular
input that the LU kernels detect and report; after it, every kernel still reads
in-bounds pivot indices.  The timeout is forced by the wait_polls parameter,
which makes the first barrier wait give up without polling; the CTA then waits
(with the long drain limit) for the products it already issued, frees its tensor
memory and returns.  After each failure the same process factors and solves a
normal problem, so the CUDA context is still usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import rss as orss
from oracle.dense import relres
from oracle.rss import KernelSpec

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15458_gb300 as P
    return P


def _still_works(P, side=32):
    pts = W.grid_points(side)
    f = P.rss_factor(P.rss_build_tree(pts, 16), kind=P.LAPLACE, eps=1e-8, h=1 / side)
    b = W.gaussian_rhs(side * side, 1, False, 3)
    x = torch.from_numpy(b[:, 0].copy()).cuda()
    P.rss_solve(f, x)
    torch.cuda.synchronize()
    assert relres(pts, KernelSpec("laplace", h=1 / side), x.cpu().numpy()[:, None], b) <= 1e-7


@pytest.mark.parametrize("side,where", [(64, "elimination"), (16, "top")])
def test_zero_matrix_returns_enumeric(P, side, where):
    """A = 0 (the real polynomial test kernel with no terms and a zero diagonal).
    With leaf 64 on a 64 x 64 grid every leaf box has k = 0 (its proxy stack is
    zero) and X_RR = 0, so the LU of the first box stops at a zero pivot; on a
    16 x 16 grid there is no compressed level and the dense top LU meets it.  The
    oracle rejects the same matrix."""
    pts = W.grid_points(side)
    spec = KernelSpec("rpoly", h=1 / side, coef=(), scale=1.0, diag=0.0)
    with pytest.raises(np.linalg.LinAlgError):
        orss.factor(pts, spec, 1e-6, leaf=64)
    tree = P.rss_build_tree(pts, 64)
    with pytest.raises(P.RSSError, match="ENUMERIC") as ei:
        P.rss_factor(tree, kind=P.TEST_RPOLY, eps=1e-6, h=1 / side, coef=(), diag=0.0)
    assert ei.value.status == 4
    assert ("top" in str(ei.value)) == (where == "top")
    _still_works(P)


@pytest.mark.parametrize("kind,side", [("laplace", 64), ("helmholtz", 64), ("laplace", 256)])
def test_schur_barrier_timeout_returns_etimeout(P, kind, side):
    """wait_polls = -1 makes the first barrier wait of the tensor-core Schur update
    (real: k_schur_tc, and at 256 x 256 the row-block form k_schur_tc_rows, which
    then has two tiles of products in flight; complex: k_schur_tc_c) give up at
    once: rss_factor must return RSS_ETIMEOUT, and a factorization with the default
    limit must then succeed in the same process and give the oracle's ranks."""
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    kw = dict(kind=P.LAPLACE if kind == "laplace" else P.HELMHOLTZ, eps=1e-6, h=1 / side, kappa=25.0)
    with pytest.raises(P.RSSError, match="ETIMEOUT") as ei:
        P.rss_factor(tree, wait_polls=-1, **kw)
    assert ei.value.status == 5
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_factor(tree, wait_polls=-2, **kw)
    f = P.rss_factor(tree, **kw)
    if side == 64:
        fac = orss.factor(pts, KernelSpec(kind, h=1 / side, kappa=25.0), 1e-6, leaf=64)
        for g in (8, 4):
            assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    else:
        b = W.gaussian_rhs(side * side, 1, False, 9)
        x = torch.from_numpy(b[:, 0].copy()).cuda()
        P.rss_solve(f, x)
        torch.cuda.synchronize()
        assert relres(pts, KernelSpec(kind, h=1 / side), x.cpu().numpy()[:, None], b) <= 1e-5
    _still_works(P)


def test_sweep_barrier_timeout_voids_the_result(P):
    """A grid-barrier wait of the persistent solve sweeps that runs out must not leave a
    silently wrong answer: every entry of the result becomes NaN.  wait_polls = -1
    makes every barrier wait give up at once (the factorization takes the FP64 Schur
    update, which has no bounded wait of its own); the same factorization with the
    default limit solves correctly, and the per-class form does not use the barrier."""
    side = 64
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    table = {"launch": "persistent", "spread": 1, "ctas_per_sm": 0}
    b = W.gaussian_rhs(side * side, 2, False, 5)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T
    bad = P.rss_factor(tree, kind=P.LAPLACE, eps=1e-8, h=1 / side, schur_fp64=True, wait_polls=-1,
                       tune_table=table)
    x = bt.clone()
    P.rss_solve(bad, x)
    torch.cuda.synchronize()
    assert bool(torch.isnan(x).all())
    good = P.rss_factor(tree, kind=P.LAPLACE, eps=1e-8, h=1 / side, schur_fp64=True, tune_table=table)
    for f in (good, P.rss_factor(tree, kind=P.LAPLACE, eps=1e-8, h=1 / side, schur_fp64=True, wait_polls=-1,
                                 tune_table={"launch": "per_class"})):
        x = bt.clone()
        P.rss_solve(f, x)
        torch.cuda.synchronize()
        assert relres(pts, KernelSpec("laplace", h=1 / side), x.cpu().numpy(), b) <= 1e-7
    _still_works(P)
