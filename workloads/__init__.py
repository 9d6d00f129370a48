"""Seeded synthetic inputs for strong recursive skeletonization (RS-S) runs.

This module holds no RS-S arithmetic: it only makes the point sets and the
right-hand sides that both the CPU oracle and the CUDA path consume, so that
the two sides see byte-identical inputs.

Points are the cell centres of a uniform side x side grid on [0,1]^2
(Section 5: piecewise-constant collocation on a uniform grid, h = 1/sqrt(N)).
User order is row-major: index = iy * side + ix.
"""
from __future__ import annotations

import numpy as np

LAPLACE = 0
HELMHOLTZ = 1
HELMHOLTZ_LS = 4   # symmetrised Lippmann-Schwinger (the paper's Helmholtz problem)


def grid_points(side: int) -> np.ndarray:
    """(side*side, 2) float64 cell centres ((ix+1/2)h, (iy+1/2)h), h = 1/side."""
    h = 1.0 / side
    iy, ix = np.divmod(np.arange(side * side, dtype=np.int64), side)
    pts = np.empty((side * side, 2), dtype=np.float64)
    pts[:, 0] = (ix + 0.5) * h
    pts[:, 1] = (iy + 0.5) * h
    return pts


def gaussian_rhs(n: int, nrhs: int, is_complex: bool, seed: int) -> np.ndarray:
    """(n, nrhs) N(0,1) entries (complex: re and im iid N(0,1)), numpy PCG64."""
    rng = np.random.default_rng(seed)
    if is_complex:
        b = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    else:
        b = rng.standard_normal((n, nrhs))
    return np.asfortranarray(b)


def shuffled(points: np.ndarray, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """A seeded permutation of the points (to exercise user-order handling)."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(points.shape[0])
    return points[p].copy(), p


# The workloads, named by what they are.  kind, side, dtype, eps, nrhs, seed.
WORKLOADS = {
    "laplace_64x64_eps1e-8": dict(kind=LAPLACE, side=64, complex=False, kappa=0.0,
                                   eps=1e-8, nrhs=1, seed=1000),
    "helmholtz_k25_256x256_eps1e-6": dict(kind=HELMHOLTZ, side=256, complex=True,
                                           kappa=25.0, eps=1e-6, nrhs=16, seed=1001),
    "laplace_256x256_eps1e-6": dict(kind=LAPLACE, side=256, complex=False, kappa=0.0,
                                     eps=1e-6, nrhs=1, seed=1003),
    "laplace_512x512_eps1e-6": dict(kind=LAPLACE, side=512, complex=False, kappa=0.0,
                                     eps=1e-6, nrhs=1, seed=1005),
    "laplace_1024x1024_eps1e-6": dict(kind=LAPLACE, side=1024, complex=False, kappa=0.0,
                                       eps=1e-6, nrhs=1, seed=1002),
    "helmholtz_k50_2048x2048_eps1e-6": dict(kind=HELMHOLTZ, side=2048, complex=True,
                                             kappa=50.0, eps=1e-6, nrhs=64, seed=1004),
}
# All workloads: leaf boxes of 64 points (8x8), 64 proxy points on a circle of
# radius 2.5 x box half-width, diagonal entries A_ii = 1.
LEAF = 64
PROXY_N = 64
PROXY_RADIUS_OVER_SIDE = 1.25
