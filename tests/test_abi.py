"""The C-ABI library builds, loads and exports every entry point of include/rss.h.

Host-only calls (tree construction and its argument checks) run without a GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_15458_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rss_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"rss_build_tree", "rss_factor", "rss_solve", "rss_free"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_tree_validation_on_host():
    import paper_2310_15458_gb300 as P
    t = P.rss_build_tree(W.grid_points(64), 64)
    assert t.n == 4096
    pts, _ = W.shuffled(W.grid_points(32), 1)
    assert P.rss_build_tree(pts, 16).n == 1024
    bad = [W.grid_points(64)[:-1], W.grid_points(64) * np.array([1.0, 2.0])]
    for b in bad:
        with pytest.raises(P.RSSError, match="EINVAL"):
            P.rss_build_tree(b, 64)
    dup = W.grid_points(16)
    dup[1] = dup[0]
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_build_tree(dup, 16)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_build_tree(W.grid_points(24), 64)     # 24 / 8 = 3 is not a power of two


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    import paper_2310_15458_gb300.rss as R
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        R._load()


def test_self_integral_is_host_only_and_matches_oracle():
    """rss_self_integral (Eqs. 16, 20) runs on the host: the Laplace closed form and
    the Helmholtz Gauss-Legendre reduction against the oracle's adaptive quadrature."""
    import paper_2310_15458_gb300 as P
    from oracle.rss import self_integral
    for h in (1 / 64, 1 / 1024):
        assert abs(P.rss_self_integral(P.LAPLACE, h) - self_integral("laplace", h)) <= \
            1e-13 * abs(self_integral("laplace", h))
        for kappa in (25.0, 50.0):
            o = self_integral("helmholtz", h, kappa)
            assert abs(P.rss_self_integral(P.HELMHOLTZ, h, kappa) - o) <= 1e-12 * abs(o)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_self_integral(P.HELMHOLTZ, 1 / 64, 0.0)


def test_binding_refuses_overlapping_columns(lib):
    """A right-hand-side matrix whose columns share storage (an expanded tensor, a
    broadcast array: stride < n) or that cannot be written is refused by the
    binding before anything reaches the library, which would otherwise read and
    write n * nrhs entries through it."""
    import torch

    import paper_2310_15458_gb300 as P
    n = 256
    fake = P.rss.Factor(None, n, False, None)     # never passed to the library
    b = torch.ones(n, 1, dtype=torch.float64).expand(n, 4)
    assert b.stride() == (1, 0)
    with pytest.raises(ValueError, match="overlap"):
        P.rss_solve(fake, b)
    short = torch.zeros(4, n - 1, dtype=torch.float64).T   # stride n - 1 < n
    with pytest.raises(ValueError, match="wrong number of rows"):
        P.rss_solve(fake, short)
    rows = torch.zeros(2 * n, 3, dtype=torch.float64)[::2]   # stride(0) = 2
    with pytest.raises(ValueError, match="column-major"):
        P.rss_solve(fake, rows)
    arr = np.broadcast_to(np.ones((n, 1)), (n, 4))
    with pytest.raises(ValueError):
        P.rss_solve(fake, arr)
    overl = np.lib.stride_tricks.as_strided(np.zeros(n + 8), shape=(n, 4), strides=(8, 16))
    with pytest.raises(ValueError, match="overlap"):
        P.rss_solve(fake, overl)
    # one column may carry any stride along its unused second axis
    one = torch.zeros(1, n, dtype=torch.float64).T
    assert P.rss._columns(one, n, "b") == (1, n)
