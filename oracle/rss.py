"""Plain CPU restatement of strong recursive skeletonization (RS-S).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): never imported by the
product path.

Every step follows the paper's order and notation:

* kernel matrix A_ij = K(x_i, x_j) for i != j, Eq. (3); Laplace kernel
  Eq. (14)/(15), Helmholtz kernel Eq. (18);
* perfect quadtree, near field N(B) and far field F(B), Section 2.1;
  distance-2 neighbours M(B) = N(N(B)) minus N(B) and B, Definition 2;
* column interpolative decomposition, Definition 1, by column-pivoted
  Householder QR (the greedy choice of Section 2.2) of the proxy-compressed
  stack [A_MB; K_PB; A_BM^*; K_BP^*], Eqs. (4), (5) and (6);
* sparsification S, Eq. (7), LU of X_RR and block elimination, Eq. (8);
* the per-box operator Z(A; B) = V A W, Eq. (9); the box sweep of Eq. (10);
  merging of children's skeletons at the parent level (Fig. "merge");
  Algorithm 1 level loop L .. 1;
* solve: upward then downward traversal, Section 2.5.

Readings where the paper is silent (each also listed in the design notes):
  - boxes of a level are visited colour-major with colour (ix mod 3) +
    3 (iy mod 3), row-major within a colour (Algorithm 1 asks only for "a
    given ordering"; same-colour boxes are more than distance 2 apart, so they
    touch disjoint blocks, Section 3);
  - ID truncation: Frobenius norm, stop at the first k with
    ||R22||_F <= eps ||Y||_F (then ||Y_R - Y_S T||_F = ||R22||_F, Definition 1);
  - pivot ties: columns whose remaining squared norm is within rounding noise
    of the maximum (1e-6 relative, plus 1e-12 sqrt(max x largest initial
    squared norm)) count as tied, and the lowest original column wins;
  - downdated column norms are re-accumulated once they fall below
    sqrt(unit roundoff) of their last accumulated value (LAPACK's rule);
  - compression on box grids of side >= 4, a dense LU on what remains at
    side 2 (there is no far field at the two top levels);
  - children are merged in the order SW, SE, NW, NE, each child's skeleton in
    pivot order;
  - LU of X_RR with partial pivoting (largest modulus, lowest row on ties).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import special

# Pivot ties.  A remaining squared column norm n_c carries rounding noise of
# about eps_mach ||x_c|| ||y_c|| (trailing column x_c, original column y_c), so
# columns with n_c >= n_max - (TIE_REL n_max + TIE_ABS sqrt(n_max y2max)), y2max
# the largest initial squared column norm, cannot be told apart and count as
# tied (exact-arithmetic ties from the grid's symmetry show up as such
# rounding-level differences).
TIE_REL = 1e-6
TIE_ABS = 1e-12
# A downdated squared column norm is re-accumulated from the trailing rows once
# it has fallen below this fraction of the value it was last accumulated at
# (sqrt of the unit roundoff, LAPACK geqp3's threshold).  Between
# re-accumulations a downdated value is therefore accurate to about
# eps_mach / RECOMPUTE_REL = 7e-9 relative per downdate (a few 1e-8 after many
# steps), well inside the 1e-6 tie window above.
RECOMPUTE_REL = 1.4901161193847656e-08


# ---------------------------------------------------------------------------
# Kernels (Eqs. 3, 14, 15, 18)
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class KernelSpec:
    """Entries of A.

    kind: 'laplace'   A_ij = -(h^2 / 2 pi) log |x_i - x_j|            (Eq. 15)
          'helmholtz' A_ij = h^2 (i/4) H0^(1)(kappa |x_i - x_j|)      (Eq. 18 with
                      the scaling of the dense-solver workloads: no kappa^2 b factor)
          'ls'        Lippmann-Schwinger (Eq. 19): A_ij = w_i w_j h^2 (i/4) H0^(1)(kappa r)
                      with w = kappa sqrt(b(x)), A_ii = 1 + w_i^2 diag (Eq. 20 when diag
                      is the self-cell integral of (i/4) H0^(1)); proxy points (Eq. 6)
                      take the weight kappa (sqrt(b) = 1)
          'poly'      A_ij = scale * conj(w_i) w_j sum_d coef[d] (z_i - z_j)^d, z = x + i y,
                      w = exp(i (phase[0] x + phase[1] y)): a test kernel whose far
                      field is exactly low rank, so that RS-S is exact up to
                      rounding (used to pin the bookkeeping, never a workload)
          'rpoly'     real part of 'poly' with no phase weights
    diag: A_ii.
    """
    kind: str
    h: float
    kappa: float = 0.0
    diag: complex = 1.0
    coef: tuple = ()
    scale: float = 1.0
    phase: tuple = (0.0, 0.0)
    bump: tuple = (0.5, 0.5, 32.0)   # 'ls': b(x) = exp(-bump[2] |x - (bump[0], bump[1])|^2)

    @property
    def is_complex(self) -> bool:
        return self.kind in ("helmholtz", "poly", "ls")

    @property
    def dtype(self):
        return np.complex128 if self.is_complex else np.float64


def ls_weights(spec: KernelSpec, X: np.ndarray) -> np.ndarray:
    """w = kappa sqrt(b(x)) of the symmetrised Lippmann-Schwinger equation (Eq. 19)."""
    cx, cy, a = spec.bump
    return spec.kappa * np.exp(-0.5 * a * ((X[:, 0] - cx) ** 2 + (X[:, 1] - cy) ** 2))


def self_integral(kind: str, h: float, kappa: float = 0.0) -> complex:
    """Integral of the kernel over the self cell [-h/2, h/2]^2 (Eqs. 16 and 20).

    By the cell's eight-fold symmetry the integral is 8 times the integral over
    the triangle 0 <= theta <= pi/4, 0 <= rho <= a / cos(theta), a = h/2:
      Laplace:   int_0^R rho log(rho) drho = R^2 log(R)/2 - R^2/4, integrated in
                 theta in closed form: -(1/2pi) 2 a^2 (2 log a + log 2 - 3 + pi/2);
      Helmholtz: int_0^R rho H0(kappa rho) drho = R H1(kappa R)/kappa + 2i/(pi kappa^2)
                 (the limit at 0 from Y1(z) ~ -2/(pi z)), integrated in theta by
                 adaptive quadrature.
    """
    a = 0.5 * h
    if kind == "laplace":
        return -(1.0 / (2.0 * np.pi)) * 2.0 * a * a * (2.0 * np.log(a) + np.log(2.0) - 3.0 + 0.5 * np.pi)
    if kind in ("helmholtz", "ls"):
        from scipy.integrate import quad

        def f(t, part):
            R = a / np.cos(t)
            v = R * special.hankel1(1, kappa * R) / kappa + 2j / (np.pi * kappa * kappa)
            return v.real if part == 0 else v.imag
        re = quad(f, 0.0, 0.25 * np.pi, args=(0,), epsabs=0.0, epsrel=1e-13, limit=200)[0]
        im = quad(f, 0.0, 0.25 * np.pi, args=(1,), epsabs=0.0, epsrel=1e-13, limit=200)[0]
        return 8.0 * 0.25j * complex(re, im)
    raise ValueError(f"no self integral for kernel kind {kind!r}")


def kernel_block(spec: KernelSpec, X1: np.ndarray, X2: np.ndarray, proxy1: bool = False,
                 proxy2: bool = False) -> np.ndarray:
    """K(x_a, y_b) for all rows a of X1 and b of X2 (no diagonal rule).

    proxy1 / proxy2: the points of X1 / X2 are proxy points (they take the
    weight kappa for 'ls')."""
    if spec.kind == "ls":
        base = KernelSpec("helmholtz", spec.h, spec.kappa)
        K = kernel_block(base, X1, X2)
        w1 = np.full(X1.shape[0], spec.kappa) if proxy1 else ls_weights(spec, X1)
        w2 = np.full(X2.shape[0], spec.kappa) if proxy2 else ls_weights(spec, X2)
        return K * w1[:, None] * w2[None, :]
    dx = X1[:, None, 0] - X2[None, :, 0]
    dy = X1[:, None, 1] - X2[None, :, 1]
    if spec.kind == "laplace":
        r = np.hypot(dx, dy)
        return -(spec.h * spec.h / (2.0 * np.pi)) * np.log(r)
    if spec.kind == "helmholtz":
        r = np.hypot(dx, dy)
        return (spec.h * spec.h) * (0.25j) * special.hankel1(0, spec.kappa * r)
    if spec.kind in ("poly", "rpoly"):
        z = dx + 1j * dy
        acc = np.zeros(z.shape, dtype=np.complex128)
        for d, c in enumerate(spec.coef):
            acc += c * z ** d
        acc *= spec.scale
        if spec.kind == "rpoly":
            return acc.real.copy()
        w1 = np.exp(1j * (spec.phase[0] * X1[:, 0] + spec.phase[1] * X1[:, 1]))
        w2 = np.exp(1j * (spec.phase[0] * X2[:, 0] + spec.phase[1] * X2[:, 1]))
        return acc * w1.conj()[:, None] * w2[None, :]
    raise ValueError(f"unknown kernel kind {spec.kind!r}")


def entries(spec: KernelSpec, X: np.ndarray, I: np.ndarray, J: np.ndarray) -> np.ndarray:
    """A[I, J] for global index arrays I, J: kernel off the diagonal, spec.diag on it (Eq. 3)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        A = kernel_block(spec, X[I], X[J]).astype(spec.dtype, copy=False)
    same = I[:, None] == J[None, :]
    if same.any():
        A = np.array(A, copy=True)
        if spec.kind == "ls":
            w = ls_weights(spec, X[I])
            A[same] = (1.0 + w * w * spec.diag)[np.nonzero(same)[0]]
        else:
            A[same] = spec.diag
    return A


# ---------------------------------------------------------------------------
# Interpolative decomposition by column-pivoted QR (Definition 1, Section 2.2)
# ---------------------------------------------------------------------------
def _abs2(a):
    return a.real * a.real + a.imag * a.imag if np.iscomplexobj(a) else a * a


def cpqr_id(Y: np.ndarray, eps: float):
    """Column ID of Y: Y[:, R] ~= Y[:, S] T with ||Y_R - Y_S T||_F <= eps ||Y||_F.

    Householder QR with column pivoting (Businger-Golub greedy rule): at step j
    the remaining column of largest 2-norm is moved to position j, a reflector
    H = I - tau v v^H (v_0 = 1) zeroes it below the diagonal, and the trailing
    columns' norms are downdated.  Truncation at the first k whose trailing
    block R22 has ||R22||_F <= eps ||Y||_F.  T = R11^{-1} R12 by back
    substitution.

    Returns (k, perm, T, R): S = perm[:k], R-set = perm[k:] (positions into the
    columns of Y), T of shape (k, n-k), and the triangular factor.
    """
    R = np.array(Y, dtype=np.complex128 if np.iscomplexobj(Y) else np.float64, copy=True)
    m, n = R.shape
    perm = np.arange(n)
    norm2 = _abs2(R).sum(axis=0)
    ref = norm2.copy()
    y2max = norm2.max() if n else 0.0
    thresh = eps * eps * norm2.sum()
    k = 0
    kmax = min(m, n)
    while k < kmax:
        if norm2[k:].sum() <= thresh:
            break
        rem = norm2[k:]
        mx = rem.max()
        cand = k + np.flatnonzero(rem >= mx - (TIE_REL * mx + TIE_ABS * np.sqrt(mx * y2max)))
        p = int(cand[np.argmin(perm[cand])])
        if p != k:
            R[:, [k, p]] = R[:, [p, k]]
            perm[[k, p]] = perm[[p, k]]
            norm2[[k, p]] = norm2[[p, k]]
            ref[[k, p]] = ref[[p, k]]
        x = R[k:, k]
        alpha = np.sqrt(_abs2(x).sum())
        if alpha == 0.0:          # stale norm: the column is already zero
            break
        x0 = x[0]
        ax0 = abs(x0)
        phase = x0 / ax0 if ax0 != 0.0 else 1.0
        beta = -phase * alpha
        v = x / (x0 - beta)
        v[0] = 1.0
        tau = (alpha + ax0) / alpha
        if k + 1 < n:
            tr = R[k:, k + 1:]
            w = v.conj() @ tr
            tr -= tau * np.outer(v, w)
        R[k, k] = beta
        R[k + 1:, k] = 0.0
        k += 1
        if k < n:
            norm2[k:] -= _abs2(R[k - 1, k:])
            stale = np.flatnonzero(norm2[k:] < RECOMPUTE_REL * ref[k:]) + k
            for c in stale:
                norm2[c] = _abs2(R[k:, c]).sum()
                ref[c] = norm2[c]
    T = upper_solve(R[:k, :k], R[:k, k:])
    return k, perm, T, R


def upper_solve(U: np.ndarray, B: np.ndarray) -> np.ndarray:
    """U^{-1} B for upper-triangular U, by back substitution."""
    k = U.shape[0]
    X = np.array(B, dtype=np.result_type(U, B), copy=True)
    for i in range(k - 1, -1, -1):
        if i + 1 < k:
            X[i] -= U[i, i + 1:] @ X[i + 1:]
        X[i] /= U[i, i]
    return X


# ---------------------------------------------------------------------------
# LU with partial pivoting (the LU of X_RR in Eq. 8, and the top dense block)
# ---------------------------------------------------------------------------
def lu_factor_pp(A: np.ndarray):
    """P A = L U, right-looking, pivot = largest modulus in the column (lowest row on ties).

    Returns (LU, piv) with L unit-lower and U upper packed in LU, and piv[j] the
    row exchanged with row j at step j (LAPACK getrf convention, 0-based).
    """
    LU = np.array(A, copy=True)
    n = LU.shape[0]
    piv = np.arange(n)
    for j in range(n):
        p = j + int(np.argmax(_abs2(LU[j:, j])))
        if LU[p, j] == 0:
            raise np.linalg.LinAlgError("singular block in LU")
        if p != j:
            LU[[j, p]] = LU[[p, j]]
        piv[j] = p
        LU[j + 1:, j] /= LU[j, j]
        LU[j + 1:, j + 1:] -= np.outer(LU[j + 1:, j], LU[j, j + 1:])
    return LU, piv


def apply_row_swaps(piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """P B for the getrf-style pivot vector."""
    B = np.array(B, copy=True)
    for j, p in enumerate(piv):
        if p != j:
            B[[j, p]] = B[[p, j]]
    return B


def unit_lower_solve(LU: np.ndarray, B: np.ndarray) -> np.ndarray:
    """L^{-1} B with L the unit-lower part of LU (forward substitution)."""
    X = np.array(B, dtype=np.result_type(LU, B), copy=True)
    n = LU.shape[0]
    for i in range(1, n):
        X[i] -= LU[i, :i] @ X[:i]
    return X


def right_upper_solve(X: np.ndarray, LU: np.ndarray) -> np.ndarray:
    """X U^{-1} with U the upper part of LU (column by column)."""
    E = np.array(X, dtype=np.result_type(X, LU), copy=True)
    r = LU.shape[0]
    for j in range(r):
        if j:
            E[:, j] -= E[:, :j] @ LU[:j, j]
        E[:, j] /= LU[j, j]
    return E


def lu_solve_pp(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^{-1} B from lu_factor_pp."""
    Y = unit_lower_solve(LU, apply_row_swaps(piv, B))
    return upper_solve(np.triu(LU), Y)


# ---------------------------------------------------------------------------
# Quadtree (Section 2.1)
# ---------------------------------------------------------------------------
@dataclass
class Grid:
    side: int            # points per grid row
    x0: float            # coordinates of the first cell centre
    y0: float
    hg: float            # grid spacing
    ix: np.ndarray       # integer grid coordinates of each user point
    iy: np.ndarray


def grid_of(points: np.ndarray) -> Grid:
    n = points.shape[0]
    side = int(round(np.sqrt(n)))
    if side * side != n:
        raise ValueError("points must form a square uniform grid")
    x0, y0 = points[:, 0].min(), points[:, 1].min()
    hg = (points[:, 0].max() - x0) / (side - 1) if side > 1 else 1.0
    ix = np.rint((points[:, 0] - x0) / hg).astype(np.int64)
    iy = np.rint((points[:, 1] - y0) / hg).astype(np.int64)
    if (ix.min() < 0 or ix.max() >= side or iy.min() < 0 or iy.max() >= side
            or np.unique(iy * side + ix).size != n):
        raise ValueError("points must form a square uniform grid")
    return Grid(side, x0, y0, hg, ix, iy)


def chebyshev(b1, b2, g):
    return max(abs(b1 % g - b2 % g), abs(b1 // g - b2 // g))


def ring(b, g, dist):
    """Boxes at Chebyshev distance exactly `dist` from box b (row-major offsets, in-grid)."""
    bx, by = b % g, b // g
    out = []
    for dy in range(-dist, dist + 1):
        for dx in range(-dist, dist + 1):
            if max(abs(dx), abs(dy)) != dist:
                continue
            x, y = bx + dx, by + dy
            if 0 <= x < g and 0 <= y < g:
                out.append(y * g + x)
    return out


def stencil(b, g):
    """All boxes at Chebyshev distance <= 2 from b (including b)."""
    bx, by = b % g, b // g
    return [y * g + x for y in range(max(0, by - 2), min(g, by + 3))
            for x in range(max(0, bx - 2), min(g, bx + 3))]


def colour_order(g):
    """Colour-major, row-major within a colour; colour = (ix mod 3) + 3 (iy mod 3)."""
    boxes = []
    for c in range(9):
        cx, cy = c % 3, c // 3
        boxes += [by * g + bx for by in range(cy, g, 3) for bx in range(cx, g, 3)]
    return boxes


def children(P, g_parent):
    """Children of parent P in the order SW, SE, NW, NE (y grows northwards)."""
    px, py = P % g_parent, P // g_parent
    gc = 2 * g_parent
    return [(2 * py + cy) * gc + (2 * px + cx) for cy in (0, 1) for cx in (0, 1)]


def proxy_points(centre, radius, nproxy):
    th = 2.0 * np.pi * np.arange(nproxy) / nproxy
    return np.stack([centre[0] + radius * np.cos(th), centre[1] + radius * np.sin(th)], axis=1)


# ---------------------------------------------------------------------------
# Factorization (Algorithm 1)
# ---------------------------------------------------------------------------
@dataclass
class BoxRecord:
    side: int                 # box-grid side of the level
    box: int
    S: np.ndarray             # global indices of the skeleton points (pivot order)
    R: np.ndarray             # global indices of the redundant points
    C: np.ndarray             # global indices of S followed by the neighbours' active points
    T: np.ndarray             # k x r interpolation matrix
    LU: np.ndarray            # r x r packed LU of X_RR
    piv: np.ndarray
    E: np.ndarray             # c x r: X_CR U_R^{-1}
    F: np.ndarray             # r x c: L_R^{-1} P_R X_RC


@dataclass
class Factorization:
    n: int
    dtype: object
    records: list = field(default_factory=list)
    top_idx: np.ndarray = None
    top_LU: np.ndarray = None
    top_piv: np.ndarray = None
    ranks: dict = field(default_factory=dict)        # box-grid side -> array of k per box
    level_sizes: dict = field(default_factory=dict)  # box-grid side -> array of n_B per box


def build_proxy_stack(spec, X, blocks, pts, B, g, centre, radius, nproxy):
    """Y = [A_MB; K_PB; A_BM^*; K_BP^*] (Eq. 6 stacked as in Eq. 4)."""
    Ms = ring(B, g, 2)
    pB = pts[B]
    yp = proxy_points(centre, radius, nproxy)
    rows = [blocks[(m, B)] for m in Ms]
    rows.append(kernel_block(spec, yp, X[pB], proxy1=True).astype(spec.dtype, copy=False))
    rows += [blocks[(B, m)].conj().T for m in Ms]
    rows.append(kernel_block(spec, X[pB], yp, proxy2=True).astype(spec.dtype, copy=False).conj().T)
    return np.vstack(rows)


def sparsify(A_SS, A_SR, A_RS, A_RR, A_NS, A_NR, A_SN, A_RN, T):
    """Blocks of S^* (P^T A P) S that touch R (Eq. 7): X_CR, X_RC and X_RR, C = S u N."""
    TH = T.conj().T
    X_SR = A_SR - A_SS @ T
    X_NR = A_NR - A_NS @ T
    X_RS = A_RS - TH @ A_SS
    X_RN = A_RN - TH @ A_SN
    X_RR = A_RR - A_RS @ T - TH @ X_SR
    return np.vstack([X_SR, X_NR]), np.hstack([X_RS, X_RN]), X_RR


def eliminate(X_CR, X_RC, X_RR):
    """Eq. (8): P_R X_RR = L_R U_R, E = X_CR U_R^{-1}, F = L_R^{-1} P_R X_RC."""
    LU, piv = lu_factor_pp(X_RR)
    E = right_upper_solve(X_CR, LU)
    F = unit_lower_solve(LU, apply_row_swaps(piv, X_RC))
    return LU, piv, E, F


def skeletonize_box(spec, X, blocks, pts, B, g, eps, centre, radius, nproxy):
    """Strong_Skeletonization(B) of Algorithm 1: ID, sparsify, eliminate, update A_NN."""
    pB = pts[B]
    n = pB.size
    Y = build_proxy_stack(spec, X, blocks, pts, B, g, centre, radius, nproxy)
    k, perm, T, _ = cpqr_id(Y, eps)
    if k >= n:
        return k, None
    Sp, Rp = perm[:k], perm[k:]
    Ns = ring(B, g, 1)
    A_BB = blocks[(B, B)]
    A_NB = np.vstack([blocks[(nb, B)] for nb in Ns]) if Ns else np.zeros((0, n), spec.dtype)
    A_BN = np.hstack([blocks[(B, nb)] for nb in Ns]) if Ns else np.zeros((n, 0), spec.dtype)
    X_CR, X_RC, X_RR = sparsify(A_BB[np.ix_(Sp, Sp)], A_BB[np.ix_(Sp, Rp)],
                                A_BB[np.ix_(Rp, Sp)], A_BB[np.ix_(Rp, Rp)],
                                A_NB[:, Sp], A_NB[:, Rp], A_BN[Sp, :], A_BN[Rp, :], T)
    LU, piv, E, F = eliminate(X_CR, X_RC, X_RR)
    # Schur complement update of A_CC, C = S u N (Remark 2: only A_NN-type blocks change)
    G = E @ F
    parts = [(B, Sp)] + [(nb, np.arange(pts[nb].size)) for nb in Ns]
    offs = np.cumsum([0] + [p[1].size for p in parts])
    for a, (ba, ra) in enumerate(parts):
        for b_, (bb, cb) in enumerate(parts):
            blk = blocks[(ba, bb)]
            blk[np.ix_(ra, cb)] -= G[offs[a]:offs[a + 1], offs[b_]:offs[b_ + 1]]
    C = np.concatenate([pB[Sp]] + [pts[nb] for nb in Ns])
    rec = BoxRecord(g, B, pB[Sp].copy(), pB[Rp].copy(), C, T, LU, piv, E, F)
    # R is eliminated: B keeps only its skeleton
    for other in stencil(B, g):
        if other == B:
            blocks[(B, B)] = blocks[(B, B)][np.ix_(Sp, Sp)]
        else:
            blocks[(B, other)] = blocks[(B, other)][Sp, :]
            blocks[(other, B)] = blocks[(other, B)][:, Sp]
    pts[B] = pB[Sp]
    return k, rec


def merge_level(spec, X, blocks, pts, g):
    """Level transition: a parent owns the union of its children's skeletons.

    Parent blocks at parent distance <= 2 are gathered from stored child blocks
    where the children are at distance <= 2 and evaluated from the kernel
    otherwise (those interactions were never modified, Theorem 1).
    """
    gp = g // 2
    new_pts = [np.concatenate([pts[c] for c in children(P, gp)]) for P in range(gp * gp)]
    new_blocks = {}
    for P1 in range(gp * gp):
        for P2 in stencil(P1, gp):
            rows = []
            for c1 in children(P1, gp):
                row = []
                for c2 in children(P2, gp):
                    if chebyshev(c1, c2, g) <= 2:
                        row.append(blocks[(c1, c2)])
                    else:
                        row.append(kernel_block(spec, X[pts[c1]], X[pts[c2]]).astype(spec.dtype))
                rows.append(np.hstack(row))
            new_blocks[(P1, P2)] = np.vstack(rows)
    return new_blocks, new_pts


def factor(points: np.ndarray, spec: KernelSpec, eps: float, leaf: int = 64,
           nproxy: int = 64, proxy_radius_over_side: float = 1.25,
           stop_side: int = 0) -> Factorization:
    """Algorithm 1 (sequential factorization) on a uniform grid of points.

    stop_side: if > 0, stop after the level whose box grid has this side and
    return the partial factorization (for sampled comparisons).
    """
    X = np.asarray(points, dtype=np.float64)
    grid = grid_of(X)
    ls = int(round(np.sqrt(leaf)))
    if ls * ls != leaf or grid.side % ls:
        raise ValueError("leaf must be a square number whose side divides the grid side")
    g = grid.side // ls
    if g & (g - 1):
        raise ValueError("the leaf box grid must have a power-of-two side")
    fac = Factorization(n=X.shape[0], dtype=spec.dtype)
    # leaf boxes: points in row-major order inside each box
    lb = (grid.iy // ls) * g + (grid.ix // ls)
    local = (grid.iy % ls) * ls + (grid.ix % ls)
    order = np.lexsort((local, lb))
    pts = list(np.split(order, np.cumsum(np.bincount(lb, minlength=g * g))[:-1]))
    blocks = {}
    for b1 in range(g * g):
        for b2 in stencil(b1, g):
            blocks[(b1, b2)] = entries(spec, X, pts[b1], pts[b2])
    extent = grid.side * grid.hg
    while g >= 4:
        L = extent / g
        fac.level_sizes[g] = np.array([p.size for p in pts])
        ks = np.zeros(g * g, dtype=np.int64)
        for B in colour_order(g):
            bx, by = B % g, B // g
            centre = (grid.x0 - grid.hg / 2 + (bx + 0.5) * L, grid.y0 - grid.hg / 2 + (by + 0.5) * L)
            k, rec = skeletonize_box(spec, X, blocks, pts, B, g, eps, centre,
                                     proxy_radius_over_side * L, nproxy)
            ks[B] = k
            if rec is not None:
                fac.records.append(rec)
        fac.ranks[g] = ks
        if stop_side and g == stop_side:
            return fac
        blocks, pts = merge_level(spec, X, blocks, pts, g)
        g //= 2
    # dense top: everything still active (no far field at the two top levels)
    top = np.concatenate(pts)
    nb = len(pts)
    bounds = np.cumsum([0] + [p.size for p in pts])
    A_top = np.zeros((top.size, top.size), dtype=spec.dtype)
    for b1 in range(nb):
        for b2 in range(nb):
            A_top[bounds[b1]:bounds[b1 + 1], bounds[b2]:bounds[b2 + 1]] = blocks[(b1, b2)]
    fac.top_idx = top
    fac.top_LU, fac.top_piv = lu_factor_pp(A_top)
    return fac


# ---------------------------------------------------------------------------
# Solve (Section 2.5)
# ---------------------------------------------------------------------------
def solve(fac: Factorization, b: np.ndarray) -> np.ndarray:
    """x ~= A^{-1} b: apply V_1 .. V_K (upward), the top LU, then W_K .. W_1 (downward).

    V = L S^* P^T: b_R -= T^* b_S, b_R <- L_R^{-1} P_R b_R, b_C -= E b_R.
    W = P S U:     y_R <- U_R^{-1} (y_R - F y_C),  y_S -= T y_R.
    """
    x = np.array(b, dtype=np.result_type(b, fac.dtype), copy=True)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    for rec in fac.records:
        bR = x[rec.R] - rec.T.conj().T @ x[rec.S]
        bR = unit_lower_solve(rec.LU, apply_row_swaps(rec.piv, bR))
        x[rec.R] = bR
        x[rec.C] -= rec.E @ bR
    x[fac.top_idx] = lu_solve_pp(fac.top_LU, fac.top_piv, x[fac.top_idx])
    for rec in reversed(fac.records):
        yR = x[rec.R] - rec.F @ x[rec.C]
        yR = upper_solve(np.triu(rec.LU), yR)
        x[rec.R] = yR
        x[rec.S] -= rec.T @ yR
    return x[:, 0] if squeeze else x
