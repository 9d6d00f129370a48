"""rss_solve_noalloc, the solve entry point that allocates no device memory.

It serves callers that cannot allocate at call time (a framework allocator
holding the device's memory, a latency-bound serving loop).  Its results must
equal rss_solve's; it is called twice in a row on the same factorization, with
different right-hand sides and column counts, to show that what one call leaves
in the shared scratch array does not leak into the next.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15458_gb300 as P
    return P


def _cols(b):
    return torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T   # (n, nrhs) column-major


@pytest.mark.parametrize("kind,side,leaf", [(0, 64, 64), (1, 32, 16)], ids=["laplace-f64", "helmholtz-c128"])
def test_noalloc_matches_rss_solve_twice(P, kind, side, leaf):
    """Two calls in a row that differ: the first with 36 right-hand sides (more
    columns, and the multi-column sweep workspace), the second with 3 columns of a
    fresh b.  Whatever the first call leaves in the shared scratch array must not
    reach the second call's result; each must equal rss_solve's."""
    tree = P.rss_build_tree(W.grid_points(side), leaf)
    f = P.rss_factor(tree, kind=kind, eps=1e-8, h=1.0 / side, kappa=25.0)
    for call, (nrhs, seed) in enumerate(((36, 11), (3, 12))):
        b = W.gaussian_rhs(side * side, nrhs, kind == 1, seed)
        ref = _cols(b)
        P.rss_solve(f, ref)
        x = _cols(b)
        P.rss_solve_noalloc(f, x)
        torch.cuda.synchronize()
        ref, x = ref.cpu().numpy(), x.cpu().numpy()
        err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
        assert err <= 1e-12, (call, err)


def test_noalloc_rejects_what_it_cannot_hold(P):
    side = 64
    tree = P.rss_build_tree(W.grid_points(side), 64)
    f = P.rss_factor(tree, kind=0, eps=1e-6, h=1.0 / side)
    too_many = (16 << 20) // (8 * side * side) + 1          # one column past 16 MiB
    b = torch.ones(too_many, side * side, dtype=torch.float64, device="cuda").T
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_solve_noalloc(f, b)
    assert bool(torch.all(b == 1.0))
    with pytest.raises(TypeError):
        P.rss_solve_noalloc(f, np.ones(side * side))


def test_many_rhs_before_and_after_the_slice_cache(P):
    """With 32 or more right-hand sides the sweeps run on the tensor cores.  The
    digit slices of E and F are cached by the first rss_solve that needs them;
    rss_solve_noalloc never builds that cache, so before it exists it cuts the
    factor blocks chunk by chunk, and afterwards it reads the cache.  Both forms
    agree with one-column FP64 solves to 1e-12 and with each other."""
    side = 64
    tree = P.rss_build_tree(W.grid_points(side), 64)
    f = P.rss_factor(tree, kind=0, eps=1e-6, h=1.0 / side)
    b = W.gaussian_rhs(side * side, 36, False, 12)
    before = _cols(b)
    P.rss_solve_noalloc(f, before)           # no cache yet: per-chunk products
    after = _cols(b)
    P.rss_solve(f, after)                    # builds the cache, then uses it
    again = _cols(b)
    P.rss_solve_noalloc(f, again)            # the cache now exists
    torch.cuda.synchronize()
    before, after, again = before.cpu().numpy(), after.cpu().numpy(), again.cpu().numpy()
    assert np.array_equal(after, again)
    assert np.linalg.norm(before - after) <= 1e-12 * np.linalg.norm(after)
    for j in (0, 31, 35):
        xj = torch.from_numpy(b[:, j].copy()).cuda()
        P.rss_solve(f, xj)
        xj = xj.cpu().numpy()
        assert np.linalg.norm(after[:, j] - xj) <= 1e-12 * np.linalg.norm(xj)
