"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Element-wise comparisons on small and mid-size problems (several levels, ragged
right-hand-side chunks), exactness against a dense solve where the answer is
unique, and, at the full workload sizes in the launch configuration the bench
uses, sampled box records that the oracle recomputes one by one plus the
relative residual by FFT.

Tolerances: every quantity is FP64 / complex128.  Both sides run the same
sequence of operations on the same inputs, so integer outputs (ranks, skeleton
and redundant index sets, LU pivots) must be identical.  The interpolation
matrix T = R11^{-1} R12 comes from a triangular factor whose last kept diagonal
entry is about eps ||Y||, so cond(R11) reaches ~1/eps and rounding differences
of ~1e-16 grow to ~1e-16/eps in T and in everything computed from it (E, F,
the LU of X_RR); the bound is 100x that, max(1e-10, 1e-14 / eps), for the
records of the first compressed level.  A record of a later level is computed
from blocks that the eliminations of every earlier level have updated, each
carrying its own rounding of that size, so the bound grows by one such term per
earlier level: (1 + depth) max(1e-10, 1e-14 / eps), depth = number of
compressed levels below the record's.  Solutions agree to 1e-9 relative, and
every relative residual must be <= 10 eps (the target of the workloads).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import rss as orss
from oracle.dense import dense_matrix, fft_matvec, relres
from oracle.rss import KernelSpec

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

KIND = {"laplace": 0, "helmholtz": 1, "poly": 2, "rpoly": 3}


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15458_gb300 as P
    return P


def gpu_factor(P, pts, spec, eps, leaf, full_stack=False):
    tree = P.rss_build_tree(pts, leaf)
    return P.rss_factor(tree, kind=KIND[spec.kind], eps=eps, h=spec.h, kappa=spec.kappa,
                        diag=spec.diag, coef=spec.coef, scale=spec.scale, phase=spec.phase,
                        full_stack=full_stack)


def gpu_solve(P, f, b):
    b = np.asarray(b)
    if b.ndim == 1:
        bt = torch.from_numpy(b.copy()).cuda()
    else:   # (n, nrhs) column-major
        bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T
    P.rss_solve(f, bt)
    torch.cuda.synchronize()
    return bt.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


POLY = KernelSpec("poly", h=1 / 32, coef=(0.3, 0.5 - 0.2j, 0.7, 0.1 + 0.4j), scale=0.02, diag=1.0,
                  phase=(3.0, -2.0))
RPOLY = KernelSpec("rpoly", h=1 / 32, coef=(0.3, 0.5, -0.7, 0.4), scale=0.02, diag=1.0)


@pytest.mark.parametrize("spec", [RPOLY, POLY], ids=["real", "complex"])
def test_exact_low_rank_kernel_matches_dense_solve(P, spec):
    """Exactly low-rank far field: the GPU factorization must invert A to rounding."""
    side = 32
    pts = W.grid_points(side)
    f = gpu_factor(P, pts, spec, 1e-13, 16)
    b = W.gaussian_rhs(side * side, 3, spec.is_complex, 5)
    x = gpu_solve(P, f, b)
    A = dense_matrix(pts, spec)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12
    fac = orss.factor(pts, spec, 1e-13, leaf=16)
    for g in (8, 4):
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])


def rec_tol(eps, depth=0):
    """Bound on the relative difference of a record's floating-point blocks (see
    the module docstring); depth = compressed levels eliminated before its level."""
    return (1 + depth) * max(1e-10, 1e-14 / eps)


def _compare_records(P, f, fac, eps):
    """Every oracle box record against the GPU record of the same box."""
    n_cmp = 0
    sides = sorted({rec.side for rec in fac.records}, reverse=True)
    for rec in fac.records:
        tol = rec_tol(eps, sides.index(rec.side))
        g = P.rss_box_record(f, rec.side, rec.box)
        assert g["k"] == rec.S.size and g["r"] == rec.R.size
        assert np.array_equal(g["S"], rec.S) and np.array_equal(g["R"], rec.R)
        assert np.array_equal(g["C"], rec.C)
        assert np.array_equal(g["piv"], rec.piv)
        for key, ref in (("T", rec.T), ("LU", rec.LU), ("E", rec.E), ("F", rec.F)):
            if ref.size:
                assert rel(g[key], ref) < tol, (rec.side, rec.box, key, rel(g[key], ref))
        n_cmp += 1
    return n_cmp


@pytest.mark.parametrize("full_stack", [False, True], ids=["half-stack", "full-stack"])
def test_laplace_64x64_records_and_solution_match_oracle(P, full_stack):
    """The 64 x 64 Laplace workload (eps 1e-8): every box record and the solution.

    The oracle always compresses the full stack of Eq. 4; the GPU's default for the
    real symmetric Laplace kernel compresses its first half, which must give the same ID."""
    side, eps = 64, 1e-8
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    f = gpu_factor(P, pts, spec, eps, 64, full_stack)
    fac = orss.factor(pts, spec, eps)
    for g in (8, 4):
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    assert _compare_records(P, f, fac, eps) == len(fac.records)
    b = W.gaussian_rhs(side * side, 1, False, 1000)
    x = gpu_solve(P, f, b)
    xo = orss.solve(fac, b)
    assert rel(x, xo) < 1e-9
    assert relres(pts, spec, x, b) <= 10 * eps


def test_helmholtz_records_and_solution_match_oracle(P):
    side, eps = 32, 1e-6
    pts = W.grid_points(side)
    spec = KernelSpec("helmholtz", h=1 / side, kappa=25.0)
    f = gpu_factor(P, pts, spec, eps, 16)
    fac = orss.factor(pts, spec, eps, leaf=16)
    for g in (8, 4):
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    assert _compare_records(P, f, fac, eps) == len(fac.records)
    b = W.gaussian_rhs(side * side, 3, True, 1001)
    x = gpu_solve(P, f, b)
    assert rel(x, orss.solve(fac, b)) < 1e-9
    assert relres(pts, spec, x, b) <= 10 * eps


@pytest.mark.parametrize("kappa", [25.0, 50.0], ids=["kappa25", "kappa50"])
def test_helmholtz_leaf64_every_record_matches_oracle(P, kappa):
    """128 x 128 Helmholtz, leaf 64, eps 1e-6: every record of the levels with box
    grids 16, 8 and 4.  The merged boxes of the two coarse levels hold about 100
    points, so this reaches the complex elimination of boxes too large for the
    on-chip kernel, the complex panel products and Schur update on the tensor cores
    at full operand sizes, and the real-stack ID on thread-block clusters.
    kappa = 50 is the wavenumber of the 2048 x 2048 workload."""
    side, eps = 128, 1e-6
    pts = W.grid_points(side)
    spec = KernelSpec("helmholtz", h=1 / side, kappa=kappa)
    f = gpu_factor(P, pts, spec, eps, 64)
    fac = orss.factor(pts, spec, eps, leaf=64)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    assert max(rec.S.size + rec.R.size for rec in fac.records) > 80
    assert _compare_records(P, f, fac, eps) == len(fac.records)
    b = W.gaussian_rhs(side * side, 2, True, 1004)
    x = gpu_solve(P, f, b)
    assert rel(x, orss.solve(fac, b)) < 1e-9
    assert relres(pts, spec, x, b) <= 10 * eps


def test_laplace_256x256_every_record_matches_oracle(P):
    """256 x 256 Laplace, leaf 64, eps 1e-6: every record of all four compressed
    levels (box grids 32, 16, 8, 4).  Covers the one-CTA ID (colour classes of
    about 114 boxes), the cluster ID (28 boxes and fewer), and the real panel
    products and Schur update at n_B of about 80 to 100."""
    side, eps = 256, 1e-6
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    f = gpu_factor(P, pts, spec, eps, 64)
    fac = orss.factor(pts, spec, eps, leaf=64)
    for g in (32, 16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    assert max(rec.S.size + rec.R.size for rec in fac.records) > 80
    assert _compare_records(P, f, fac, eps) == len(fac.records)
    b = W.gaussian_rhs(side * side, 1, False, 1003)
    x = gpu_solve(P, f, b)
    assert rel(x, orss.solve(fac, b)) < 1e-9
    assert relres(pts, spec, x, b) <= 10 * eps


def test_ragged_rhs_chunks_host_buffers_and_user_order(P):
    """nrhs = 9 (a ragged chunk of 8), host-buffer solve == device solve, shuffled points."""
    side, eps = 32, 1e-6
    pts, perm = W.shuffled(W.grid_points(side), 3)
    spec = KernelSpec("laplace", h=1 / side)
    f = gpu_factor(P, pts, spec, eps, 16)
    b = W.gaussian_rhs(side * side, 9, False, 44)
    x_dev = gpu_solve(P, f, b)
    x_host = np.asfortranarray(b.copy())
    P.rss_solve(f, x_host)
    assert np.array_equal(x_dev, x_host)
    for j in range(9):                     # column j alone gives the same column
        xj = gpu_solve(P, f, np.ascontiguousarray(b[:, j]))
        assert np.array_equal(xj, x_dev[:, j])
    f0 = gpu_factor(P, W.grid_points(side), spec, eps, 16)
    x0 = gpu_solve(P, f0, b[np.argsort(perm)])
    assert np.array_equal(x0[perm], x_dev)
    assert relres(pts, spec, x_dev, b) <= 10 * eps


def test_tensor_core_sweeps_many_rhs(P):
    """40 right-hand sides (a full chunk of 32 and a ragged one) take the tensor-core
    sweeps: they agree with one-column FP64 solves to 1e-12, a column's result does
    not depend on the other columns (bitwise), and the residual meets 10 eps."""
    side, eps = 64, 1e-6
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    f = gpu_factor(P, pts, spec, eps, 64)
    b = W.gaussian_rhs(side * side, 40, False, 45)
    x = gpu_solve(P, f, b)
    for j in (0, 17, 31, 32, 39):
        xj = gpu_solve(P, f, np.ascontiguousarray(b[:, j]))
        assert np.linalg.norm(x[:, j] - xj) <= 1e-12 * np.linalg.norm(xj)
    perm = np.random.default_rng(1).permutation(40)
    xp = gpu_solve(P, f, np.asfortranarray(b[:, perm]))
    assert np.array_equal(xp, x[:, perm])
    x33 = gpu_solve(P, f, np.asfortranarray(b[:, :33]))
    assert np.array_equal(x33, x[:, :33])
    assert relres(pts, spec, x, b) <= 10 * eps
    fac = orss.factor(pts, spec, eps)
    assert rel(x, orss.solve(fac, b)) < 1e-9


def test_per_box_form_equals_batched(P):
    """The plain per-box form (one box per launch) and the batched form (one launch per
    colour class and phase) compute the same factorization: same ranks, bitwise equal
    solutions (one-CTA ID in both, so the arithmetic is the same)."""
    side = 64
    tree = P.rss_build_tree(W.grid_points(side), 16)
    fb = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side, id_cluster=-1)
    fp = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side, id_cluster=-1, per_box=True)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(fb, g), P.rss_level_ranks(fp, g))
    b = W.gaussian_rhs(side * side, 2, False, 46)
    assert np.array_equal(gpu_solve(P, fb, b), gpu_solve(P, fp, b))
    assert P.rss_info(fp)["launches"] > 4 * P.rss_info(fb)["launches"]


@pytest.mark.parametrize("side,leaf", [(8, 64), (16, 64), (32, 16)])
def test_degenerate_trees(P, side, leaf):
    """One box, a 2 x 2 top only, and eps = 0 (no compression): all exact."""
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    f = gpu_factor(P, pts, spec, 0.0, leaf)
    b = W.gaussian_rhs(side * side, 2, False, 7)
    x = gpu_solve(P, f, b)
    xd = np.linalg.solve(dense_matrix(pts, spec), b)
    assert rel(x, xd) < 1e-12


@pytest.mark.parametrize("side,leaf,eps", [(32, 4, 1e-4), (64, 4, 1e-3), (16, 1, 1e-3)])
def test_small_leaves_every_record_matches_oracle(P, side, leaf, eps):
    """Leaf boxes of 4 points and of one point: boxes with fewer points than the ID
    CTA has warps, on thread-block clusters of 256 and of 512 threads per CTA (the
    partial-sum buffers of the cluster ID must hold one partial per warp).  Every
    record and the solution against the oracle."""
    pts = W.grid_points(side)
    spec = KernelSpec("laplace", h=1 / side)
    f = gpu_factor(P, pts, spec, eps, leaf)
    fac = orss.factor(pts, spec, eps, leaf=leaf)
    for g in fac.ranks:
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    assert _compare_records(P, f, fac, eps) == len(fac.records)
    b = W.gaussian_rhs(side * side, 2, False, 77)
    x = gpu_solve(P, f, b)
    assert rel(x, orss.solve(fac, b)) < 1e-9
    assert relres(pts, spec, x, b) <= 10 * eps


@pytest.mark.parametrize("kind,side,leaf", [("rpoly", 64, 64), ("rpoly", 64, 16), ("poly", 32, 16)])
def test_zero_far_field_gives_rank_zero_everywhere(P, kind, side, leaf):
    """A = I (the polynomial test kernels with no terms, unit diagonal): every proxy
    stack is zero, so every box has rank 0 and, once its neighbours are eliminated,
    c = 0; the parent levels hold no points at all.  Like the oracle, the
    factorization must still be exact: x = b bit for bit through the FP64 sweeps
    (3 columns), and through the tensor-core sweeps (40 columns, digit-slice
    products rounded at 2^-53 of each column's largest entry) to 1e-15."""
    pts = W.grid_points(side)
    spec = KernelSpec(kind, h=1 / side, coef=(), scale=1.0, diag=1.0)
    fac = orss.factor(pts, spec, 1e-6, leaf=leaf)
    assert all((fac.ranks[g] == 0).all() for g in fac.ranks)
    f = gpu_factor(P, pts, spec, 1e-6, leaf)
    for g in fac.ranks:
        assert np.array_equal(P.rss_level_ranks(f, g), fac.ranks[g])
    b = W.gaussian_rhs(side * side, 3, spec.is_complex, 8)
    assert np.array_equal(gpu_solve(P, f, b), b)
    b = W.gaussian_rhs(side * side, 40, spec.is_complex, 9)
    assert rel(gpu_solve(P, f, b), b) < 1e-15


def test_invalid_arguments(P):
    pts = W.grid_points(16)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_build_tree(pts[:-1], 16)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_build_tree(pts + np.array([[1e-3, 0]] + [[0, 0]] * 255), 16)
    t = P.rss_build_tree(pts, 16)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_factor(t, eps=-1.0)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_factor(t, kind=9)
    f = P.rss_factor(t, eps=1e-6)
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_solve(f, torch.zeros(0, 256, dtype=torch.float64, device="cuda").T)


# ---------------------------------------------------------------- full workload sizes
def _leaf_colour0_boxes(g, count):
    cand = [by * g + bx for by in range(0, g, 3) for bx in range(0, g, 3)]
    idx = np.linspace(0, len(cand) - 1, count).round().astype(int)
    return [cand[i] for i in idx]


def _oracle_leaf_record(pts, spec, eps, g, B, leaf=64, nproxy=64, ratio=1.25):
    """Oracle record of a first-colour leaf box: the blocks it reads are still
    pure kernel values, so they are generated here from the kernel alone."""
    grid = orss.grid_of(pts)
    ls = int(round(np.sqrt(leaf)))
    lb = (grid.iy // ls) * g + (grid.ix // ls)
    local = (grid.iy % ls) * ls + (grid.ix % ls)
    bx, by = B % g, B // g
    near = [y * g + x for y in range(max(0, by - 2), min(g, by + 3))
            for x in range(max(0, bx - 2), min(g, bx + 3))]
    ptsl = {}
    for b in near:
        idx = np.flatnonzero(lb == b)
        ptsl[b] = idx[np.argsort(local[idx])]
    blocks = {}
    for b1 in near:
        for b2 in near:
            if orss.chebyshev(b1, b2, g) <= 2:
                blocks[(b1, b2)] = orss.entries(spec, pts, ptsl[b1], ptsl[b2])
    L = grid.side * grid.hg / g
    centre = (grid.x0 - grid.hg / 2 + (bx + 0.5) * L, grid.y0 - grid.hg / 2 + (by + 0.5) * L)
    ptsd = dict(ptsl)
    k, rec = orss.skeletonize_box(spec, pts, blocks, ptsd, B, g, eps, centre, ratio * L, nproxy)
    return k, rec


FULL = [("laplace_1024x1024_eps1e-6", 3), ("helmholtz_k25_256x256_eps1e-6", 3)]


@pytest.mark.parametrize("name,nsample", FULL, ids=[n for n, _ in FULL])
def test_full_size_sampled_records_and_residual(P, name, nsample):
    w = W.WORKLOADS[name]
    side, eps = w["side"], w["eps"]
    pts = W.grid_points(side)
    spec = KernelSpec("laplace" if w["kind"] == W.LAPLACE else "helmholtz", h=1 / side, kappa=w["kappa"])
    f = gpu_factor(P, pts, spec, eps, W.LEAF)
    g = side // 8
    for B in _leaf_colour0_boxes(g, nsample):
        k, rec = _oracle_leaf_record(pts, spec, eps, g, B)
        assert P.rss_level_ranks(f, g)[B] == k
        if rec is None:
            continue
        gr = P.rss_box_record(f, g, B)
        assert np.array_equal(gr["S"], rec.S) and np.array_equal(gr["C"], rec.C)
        for key, ref in (("T", rec.T), ("LU", rec.LU), ("E", rec.E), ("F", rec.F)):
            assert rel(gr[key], ref) < rec_tol(eps), (B, key)
    b = W.gaussian_rhs(side * side, min(w["nrhs"], 2), spec.is_complex, w["seed"])
    x = gpu_solve(P, f, b)
    assert relres(pts, spec, x, b) <= 10 * eps


def test_tensor_core_schur_matches_fp64_schur(P):
    """The split-digit tensor-core Schur update agrees with the FP64 FMA kernel."""
    side, eps = 128, 1e-6
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    f_tc = P.rss_factor(tree, kind=0, eps=eps, h=1 / side)
    f_64 = P.rss_factor(tree, kind=0, eps=eps, h=1 / side, schur_fp64=True)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(f_tc, g), P.rss_level_ranks(f_64, g))
    for g, box in ((16, 0), (16, 137), (8, 27), (4, 5)):
        a, b = P.rss_box_record(f_tc, g, box), P.rss_box_record(f_64, g, box)
        assert np.array_equal(a["S"], b["S"]) and np.array_equal(a["C"], b["C"])
        for key in ("T", "E", "F", "LU"):
            assert rel(a[key], b[key]) < rec_tol(eps), (g, box, key)
    bvec = W.gaussian_rhs(side * side, 2, False, 21)
    x_tc, x_64 = gpu_solve(P, f_tc, bvec), gpu_solve(P, f_64, bvec)
    assert rel(x_tc, x_64) < 1e-12
    spec = KernelSpec("laplace", h=1 / side)
    assert relres(pts, spec, x_tc, bvec) <= 10 * eps


@pytest.mark.parametrize("kind,cluster", [("laplace", 0), ("helmholtz", 0), ("laplace", 16)],
                         ids=["laplace", "helmholtz", "laplace-16"])
def test_cluster_id_matches_single_cta_id(P, kind, cluster):
    """Spreading a box's ID over a thread-block cluster gives the same ranks, skeletons
    and solution as one CTA per box (the row sums are only regrouped).  The default
    policy takes clusters of up to 8 CTAs; id_cluster = 16 takes non-portable
    clusters of 16 CTAs of 512 threads on the 8 x 8 and 4 x 4 box levels."""
    side, eps = 64, 1e-7
    pts = W.grid_points(side)
    spec = KernelSpec(kind, h=1 / side, kappa=25.0)
    tree = P.rss_build_tree(pts, 16)
    fc = P.rss_factor(tree, kind=KIND[kind], eps=eps, h=1 / side, kappa=25.0, id_cluster=cluster)
    f1 = P.rss_factor(tree, kind=KIND[kind], eps=eps, h=1 / side, kappa=25.0, id_cluster=-1)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(fc, g), P.rss_level_ranks(f1, g))
    fac = orss.factor(pts, spec, eps, leaf=16)
    for rec in fac.records[::max(1, len(fac.records) // 6)]:
        a, b = P.rss_box_record(fc, rec.side, rec.box), P.rss_box_record(f1, rec.side, rec.box)
        assert np.array_equal(a["S"], b["S"])
        assert rel(a["T"], b["T"]) < rec_tol(eps)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(fc, g), fac.ranks[g])
    bvec = W.gaussian_rhs(side * side, 2, spec.is_complex, 31)
    x = gpu_solve(P, fc, bvec)
    assert rel(x, orss.solve(fac, bvec)) < 1e-9


def test_tensor_core_schur_complex_matches_fp64_schur(P):
    """Complex factors: the split-digit tensor-core Schur update agrees with the FP64 kernel."""
    side, eps = 128, 1e-6
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    f_tc = P.rss_factor(tree, kind=1, eps=eps, h=1 / side, kappa=25.0)
    f_64 = P.rss_factor(tree, kind=1, eps=eps, h=1 / side, kappa=25.0, schur_fp64=True)
    for g in (16, 8, 4):
        assert np.array_equal(P.rss_level_ranks(f_tc, g), P.rss_level_ranks(f_64, g))
    for g, box in ((16, 0), (16, 137), (8, 27), (4, 5)):
        a, b = P.rss_box_record(f_tc, g, box), P.rss_box_record(f_64, g, box)
        assert np.array_equal(a["S"], b["S"]) and np.array_equal(a["C"], b["C"])
        for key in ("T", "E", "F", "LU"):
            assert rel(a[key], b[key]) < rec_tol(eps), (g, box, key)
    bvec = W.gaussian_rhs(side * side, 2, True, 23)
    x_tc, x_64 = gpu_solve(P, f_tc, bvec), gpu_solve(P, f_64, bvec)
    assert rel(x_tc, x_64) < 1e-12
    spec = KernelSpec("helmholtz", h=1 / side, kappa=25.0)
    assert relres(pts, spec, x_tc, bvec) <= 10 * eps


@pytest.mark.parametrize("side,boxes", [
    (128, ((16, 0), (16, 137), (8, 27), (4, 5))),
    (512, ((64, 0), (64, 2001), (64, 4095), (32, 300), (16, 27), (8, 5), (4, 9))),
], ids=["128", "512"])
def test_tcgen05_schur_equals_mma_sync_schur(P, side, boxes):
    """The real Schur update issued as tcgen05 products into tensor memory and the
    one on warp-level MMAs form the same exact digit-group sums and gather them
    with the same integer arithmetic, so the two factorizations agree bit for bit.
    At 128 x 128 the tcgen05 update runs one CTA per 128 x 32 tile; at 512 x 512 the
    fine levels take the row-block form (one CTA per 128 rows, walking the column
    tiles with the group sums double-buffered in tensor memory)."""
    eps = 1e-6
    tree = P.rss_build_tree(W.grid_points(side), 64)
    f_tc = P.rss_factor(tree, kind=0, eps=eps, h=1 / side)
    f_ms = P.rss_factor(tree, kind=0, eps=eps, h=1 / side, schur_mma_sync=True)
    for g in {b[0] for b in boxes}:
        assert np.array_equal(P.rss_level_ranks(f_tc, g), P.rss_level_ranks(f_ms, g))
    for g, box in boxes:
        a, b = P.rss_box_record(f_tc, g, box), P.rss_box_record(f_ms, g, box)
        for key in ("S", "C", "T", "E", "F", "LU", "piv"):
            assert np.array_equal(a[key], b[key]), (g, box, key)
    bvec = W.gaussian_rhs(side * side, 2, False, 24)
    assert np.array_equal(gpu_solve(P, f_tc, bvec), gpu_solve(P, f_ms, bvec))


def test_tensor_core_sweeps_many_rhs_complex(P):
    """Complex factors with 32 or more right-hand sides take the complex tensor-core
    sweeps (digit-slice products with shared real/imaginary scales): they agree with
    one-column FP64 solves to 1e-12, a column's result does not depend on the other
    columns, and the residual meets 10 eps.  At 256 x 256 the leaf colour classes
    (114 boxes, two column chunks) take the tensor-core sweeps, the coarser ones the
    FP64 kernels."""
    side, eps = 256, 1e-6
    pts = W.grid_points(side)
    spec = KernelSpec("helmholtz", h=1 / side, kappa=25.0)
    f = gpu_factor(P, pts, spec, eps, 64)
    b = W.gaussian_rhs(side * side, 40, True, 47)
    x = gpu_solve(P, f, b)
    for j in (0, 17, 31, 32, 39):
        xj = gpu_solve(P, f, np.ascontiguousarray(b[:, j]))
        assert np.linalg.norm(x[:, j] - xj) <= 1e-12 * np.linalg.norm(xj)
    perm = np.random.default_rng(2).permutation(40)
    xp = gpu_solve(P, f, np.asfortranarray(b[:, perm]))
    assert np.array_equal(xp, x[:, perm])
    assert relres(pts, spec, x, b) <= 10 * eps


def test_solve_schedules_give_the_same_bits(P):
    """The launch form of the FP64 sweeps (per-class kernels, or two persistent
    launches whose schedule spreads a colour class over more or fewer CTAs)
    changes the time of a solve, not its result: every form adds the same products
    in the same order.  rss_tune_solve measures the candidates and keeps the
    fastest; a tune table passed to rss_factor applies a form directly."""
    side = 128
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    b = W.gaussian_rhs(side * side, 3, False, 48)
    tables = ([{"launch": "per_class"}] +
              [{"launch": "persistent", "spread": sp, "ctas_per_sm": c} for sp, c in ((1, 2), (4, 0), (32, 4))] +
              [{"launch": "hybrid", "spread": sp, "ctas_per_sm": 0, "tail_boxes": tb} for sp, tb in ((1, 8), (4, 100))])
    xs = []
    for t in tables:
        f = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side, tune_table=t)
        info = P.rss_info(f)
        assert info["solve_launch"] == t["launch"]
        if t["launch"] != "per_class":
            assert info["solve_spread"] == t["spread"] and info["solve_ctas_per_sm"] == t["ctas_per_sm"]
        if t["launch"] == "hybrid":
            assert info["solve_tail_boxes"] == t["tail_boxes"]
        xs.append(gpu_solve(P, f, b))
        xs.append(gpu_solve(P, f, np.ascontiguousarray(b[:, 1])))
    for x in xs[2::2]:
        assert np.array_equal(x, xs[0])
    for x in xs[1::2]:
        assert np.array_equal(x, xs[0][:, 1])
    table = P.rss_tune_solve(f, 1)
    assert len(table["candidates"]) == 11 and all(c["ms"] > 0 for c in table["candidates"])
    assert P.rss_info(f)["solve_launch"] == table["launch"]
    assert min(c["ms"] for c in table["candidates"]) == table["ms"]
    assert np.array_equal(gpu_solve(P, f, b), xs[0])
    f2 = P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side, tune_table=table)
    assert P.rss_info(f2)["solve_launch"] == table["launch"]
    with pytest.raises(P.RSSError, match="EINVAL"):
        P.rss_factor(tree, kind=0, eps=1e-6, h=1 / side, tune_table={"launch": "persistent", "spread": 0})


@pytest.mark.parametrize("nrhs", [1, 5, 12])
def test_solve_schedules_give_the_same_bits_complex(P, nrhs):
    """The same property for a complex factor (Helmholtz, kappa = 25), with 1, 5 and
    12 right-hand sides (column chunks of 1, 8 and two of 8 with a ragged one): the
    per-class, persistent and hybrid forms give the same bits, and they meet the
    oracle's solution."""
    side, eps = 128, 1e-6
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    b = W.gaussian_rhs(side * side, nrhs, True, 49)
    xs = []
    for t in ({"launch": "per_class"}, {"launch": "persistent", "spread": 2, "ctas_per_sm": 0},
              {"launch": "hybrid", "spread": 1, "ctas_per_sm": 0, "tail_boxes": 20}):
        f = P.rss_factor(tree, kind=1, eps=eps, h=1 / side, kappa=25.0, tune_table=t)
        xs.append(gpu_solve(P, f, b if nrhs > 1 else np.ascontiguousarray(b[:, 0])))
    assert np.array_equal(xs[1], xs[0]) and np.array_equal(xs[2], xs[0])
    spec = KernelSpec("helmholtz", h=1 / side, kappa=25.0)
    x0 = xs[0] if nrhs > 1 else xs[0][:, None]
    assert relres(pts, spec, x0, b) <= 10 * eps


@pytest.mark.parametrize("nrhs", [1, 3])
def test_one_cta_per_box_downward_sweep_same_bits(P, nrhs):
    """At 512 x 512 the leaf colour classes (about 455 boxes) take the downward sweep
    with one CTA per box (chunks staged ahead, no partial sums in global memory); it
    adds the same sums in the same order as the chunked kernel and the persistent
    form, so the per-class and persistent solves give the same bits."""
    side, eps = 512, 1e-6
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, 64)
    b = W.gaussian_rhs(side * side, nrhs, False, 50)
    xs = []
    for t in ({"launch": "per_class"}, {"launch": "persistent", "spread": 1, "ctas_per_sm": 0}):
        f = P.rss_factor(tree, kind=0, eps=eps, h=1 / side, tune_table=t)
        xs.append(gpu_solve(P, f, b if nrhs > 1 else np.ascontiguousarray(b[:, 0])))
    assert np.array_equal(xs[0], xs[1])
    x0 = xs[0] if nrhs > 1 else xs[0][:, None]
    assert relres(pts, KernelSpec("laplace", h=1 / side), x0, b) <= 10 * eps
