"""Continuous-batching solve server: a result is the same alone and in the mix.

Requests of 1-16 right-hand sides against three resident factorizations (two
real, one complex) arrive together, so the worker packs several requests into
each panel; every result must equal rss_solve of that request on its own.

The sweeps apply the same operations to every column, and a column's result
does not depend on the other columns of its panel.  Real panels of 32 or more
columns take the tensor-core sweeps (exact digit-slice products, the accuracy
of an FP64 product) while a smaller solo request takes the FP64 sweeps, so with
the tensor-core paths enabled the match is to 1e-12 relative; with the FP64
kernels forced (schur_fp64) it is exact.
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


@pytest.mark.parametrize("fp64", [False, True], ids=["tensor-paths", "fp64-forced"])
def test_served_results_equal_solo_results(P, fp64):
    specs = [(0, 64, 64, 0.0), (0, 32, 16, 0.0), (1, 32, 16, 25.0)]
    facs = []
    for kind, side, leaf, kappa in specs:
        tree = P.rss_build_tree(W.grid_points(side), leaf)
        facs.append(P.rss_factor(tree, kind=kind, eps=1e-6, h=1.0 / side, kappa=kappa, schur_fp64=fp64))
    srv = P.rss_server_create(1 << 30, 64)
    ids = [P.rss_server_add(srv, f) for f in facs]
    rng = np.random.default_rng(3)
    reqs = []
    for q in range(48):
        j = int(rng.integers(len(facs)))
        nrhs = int(rng.integers(1, 17))
        b = W.gaussian_rhs(facs[j].n, nrhs, facs[j].is_complex, 500 + q)
        reqs.append((j, b, P.rss_server_submit(srv, ids[j], b)))
    for j, b, t in reqs:
        x, lat = P.rss_server_wait(srv, t, timeout=60.0)
        solo = np.asfortranarray(b.copy())
        P.rss_solve(facs[j], solo)
        if fp64:
            assert np.array_equal(x, solo)
        else:
            assert np.linalg.norm(x - solo) <= 1e-12 * np.linalg.norm(solo)
        assert lat > 0
    st = P.rss_server_stats(srv)
    assert st["requests"] == 48
    assert st["batches"] < 48 and st["max_requests_per_batch"] > 1
    assert st["device_bytes_in_use"] == 0
    # the real factors' slice caches (panels of up to 64 columns take the
    # tensor-core sweeps) were built by rss_server_add and charged to the budget
    assert (st["device_bytes_reserved"] > 0) == (not fp64)


def test_server_refuses_requests_beyond_its_budget(P):
    tree = P.rss_build_tree(W.grid_points(32), 16)
    f = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / 32)
    srv = P.rss_server_create(64 * 1024, 8)   # 64 KiB: panel + solve copy + workspace of 2 columns fit, 8 do not
    fid = P.rss_server_add(srv, f)
    ok = P.rss_server_submit(srv, fid, W.gaussian_rhs(1024, 2, False, 1))
    big = P.rss_server_submit(srv, fid, W.gaussian_rhs(1024, 8, False, 2))
    P.rss_server_wait(srv, ok, timeout=60.0)
    with pytest.raises(P.RSSError, match="ENOMEM"):
        P.rss_server_wait(srv, big, timeout=60.0)


def test_server_add_charges_the_slice_cache(P):
    """A real factor served with panels of 32 or more columns needs the digit-slice
    cache of its sweeps; rss_server_add builds it and charges it to the budget, and
    refuses the factorization (RSS_ENOMEM) when it does not fit.  With panels of at
    most 16 columns no cache is needed."""
    side = 64
    f = P.rss_factor(P.rss_build_tree(W.grid_points(side), 64), kind=0, eps=1e-6, h=1 / side)
    # the cache of this factor takes tens of MB; a 3-column panel and its solve
    # workspace take well under 1 MB
    small = P.rss_server_create(4 << 20, 64)
    with pytest.raises(P.RSSError, match="ENOMEM"):
        P.rss_server_add(small, f)
    narrow = P.rss_server_create(4 << 20, 16)
    fid = P.rss_server_add(narrow, f)
    assert P.rss_server_stats(narrow)["device_bytes_reserved"] == 0
    b = W.gaussian_rhs(f.n, 3, False, 9)
    x, _ = P.rss_server_wait(narrow, P.rss_server_submit(narrow, fid, b), timeout=60.0)
    solo = np.asfortranarray(b.copy())
    P.rss_solve(f, solo)
    assert np.array_equal(x, solo)
