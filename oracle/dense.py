"""Dense and FFT reference operators for checking RS-S results.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``dense_matrix``: the full A of Eq. (3) for small N.
* ``fft_matvec``: A x on a uniform grid by zero-padded 2D FFT.  The matrix is
  block-Toeplitz with Toeplitz blocks because the points lie on a uniform grid
  and the entries depend only on the displacement (Section 5 uses the same
  property to apply A by FFT).
* ``relres``: ||A x - b|| / ||b|| (Table "notations").
"""
from __future__ import annotations

import numpy as np

from .rss import KernelSpec, entries, grid_of, kernel_block, ls_weights


def dense_matrix(points: np.ndarray, spec: KernelSpec) -> np.ndarray:
    idx = np.arange(points.shape[0])
    return entries(spec, np.asarray(points, np.float64), idx, idx)


def dense_matvec(points: np.ndarray, spec: KernelSpec, x: np.ndarray) -> np.ndarray:
    return dense_matrix(points, spec) @ x


def fft_matvec(points: np.ndarray, spec: KernelSpec, x: np.ndarray) -> np.ndarray:
    """A x via the 2s x 2s circulant embedding of the displacement kernel."""
    grid = grid_of(np.asarray(points, np.float64))
    s = grid.side
    d = np.arange(-(s - 1), s)
    DX, DY = np.meshgrid(d, d)                    # DY indexes rows, DX columns
    disp = np.stack([DX.ravel() * grid.hg, DY.ravel() * grid.hg], axis=1)
    base = KernelSpec("helmholtz", spec.h, spec.kappa) if spec.kind == "ls" else spec
    with np.errstate(divide="ignore", invalid="ignore"):   # zero displacement: replaced below
        kv = kernel_block(base, disp, np.zeros((1, 2)))[:, 0].reshape(2 * s - 1, 2 * s - 1)
    kv = kv.astype(spec.dtype)
    kv[s - 1, s - 1] = 0.0                        # the diagonal is added separately
    circ = np.zeros((2 * s, 2 * s), dtype=spec.dtype)
    for iy_, dy in enumerate(d):
        circ[dy % (2 * s), d % (2 * s)] = kv[iy_, :]
    kf = np.fft.fft2(circ)
    xv = np.asarray(x)
    squeeze = xv.ndim == 1
    if squeeze:
        xv = xv[:, None]
    out = np.empty(xv.shape, dtype=np.result_type(xv, spec.dtype))
    if spec.kind == "ls":   # A = I + W (T + diag I) W, W = diag(kappa sqrt(b))   (Eqs. 19, 20)
        w = ls_weights(spec, np.asarray(points, np.float64))
        dvec = 1.0 + w * w * spec.diag
    else:
        w = np.ones(xv.shape[0])
        dvec = np.full(xv.shape[0], spec.diag)
    for j in range(xv.shape[1]):
        pad = np.zeros((2 * s, 2 * s), dtype=np.result_type(xv, spec.dtype))
        pad[grid.iy, grid.ix] = w * xv[:, j]
        y = np.fft.ifft2(kf * np.fft.fft2(pad))[:s, :s]
        y = y if np.iscomplexobj(out) else y.real
        out[:, j] = w * y[grid.iy, grid.ix] + dvec * xv[:, j]
    return out[:, 0] if squeeze else out


def relres(points: np.ndarray, spec: KernelSpec, x: np.ndarray, b: np.ndarray) -> float:
    """||A x - b||_F / ||b||_F with A applied by FFT."""
    r = fft_matvec(points, spec, x) - b
    return float(np.linalg.norm(r) / np.linalg.norm(b))
