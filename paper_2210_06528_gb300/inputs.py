"""Seeded synthetic inputs shared by the tests, the bench and the CPU oracle runs.

This module holds no arithmetic of the fitting method: it only samples test
functions on regular grids and draws seeded random numbers (numpy PCG64).
Arrays follow the library's memory convention: shape (M_{d-1}, ..., M_0) in C
order, grid axis 0 fastest.

Workloads (shapes of the paper's 1-, 2- and 3-D experiments):
  * sinc_1d:      f(x) = sin(x)/x on [-4pi, 4pi]                   (1-D sinc study, Sec. 3.1)
  * sinc_2d:      sinc(x) sinc(y) on [-4pi, 4pi]^2 + N(0, sigma)     (2-D study, Sec. 3.2)
  * gauss_3d:     sum of 16 seeded Gaussians + sin(6 pi x) cos(4 pi y) z on [0,1]^3
  * paper_2d/3d:  the closed forms of the paper's error-convergence study (Sec. 3.2.3)
  * symmetric_sinc_1d / asymmetric_sinc_1d: the 1-D overlap and clamping studies (Sec. 3.1)
  * tensor polynomials for reproduction checks.
"""
from __future__ import annotations

import numpy as np


def sinc(x):
    """Unnormalised sinc, sin(x)/x with sinc(0) = 1."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def axis_coords(M: int, lo: float, hi: float) -> np.ndarray:
    """M equispaced physical coordinates from lo to hi inclusive."""
    if M == 1:
        return np.array([lo], dtype=np.float64)
    return lo + (hi - lo) * np.arange(M, dtype=np.float64) / (M - 1)


def mesh(npts, lo, hi):
    """Coordinate arrays for a grid in the library's layout: returns a list
    [X_0, ..., X_{d-1}] each of shape (M_{d-1}, ..., M_0)."""
    d = len(npts)
    axes = [axis_coords(npts[a], lo[a], hi[a]) for a in range(d)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")  # numpy axis 0 = grid axis d-1
    return list(reversed(grids))


def sinc_1d(M: int = 1024) -> np.ndarray:
    x = axis_coords(M, -4 * np.pi, 4 * np.pi)
    return sinc(x)


def sinc_2d(M: int = 1024, noise: float = 1e-3, seed: int = 0, dtype=np.float32) -> np.ndarray:
    X, Y = mesh([M, M], [-4 * np.pi] * 2, [4 * np.pi] * 2)
    f = sinc(X) * sinc(Y)
    if noise > 0:
        rng = np.random.default_rng(seed)
        f = f + rng.normal(0.0, noise, size=f.shape)
    return f.astype(dtype)


def gauss_3d(npts=(512, 512, 512), seed: int = 0, ngauss: int = 16, dtype=np.float32,
             chunk: int = 16) -> np.ndarray:
    """Sum of ``ngauss`` seeded isotropic Gaussians (centres U[0,1]^3, sigma
    U[0.05, 0.2], amplitude 1) plus sin(6 pi x) cos(4 pi y) z on [0,1]^3.
    Built in z-slabs of ``chunk`` planes to bound host memory."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=(ngauss, 3))
    sig = rng.uniform(0.05, 0.2, size=ngauss)
    Mx, My, Mz = npts
    x = axis_coords(Mx, 0.0, 1.0)
    y = axis_coords(My, 0.0, 1.0)
    z = axis_coords(Mz, 0.0, 1.0)
    out = np.empty((Mz, My, Mx), dtype=dtype)
    gx = [np.exp(-(x - c[i, 0]) ** 2 / (2 * sig[i] ** 2)) for i in range(ngauss)]
    gy = [np.exp(-(y - c[i, 1]) ** 2 / (2 * sig[i] ** 2)) for i in range(ngauss)]
    sx = np.sin(6 * np.pi * x)
    cy = np.cos(4 * np.pi * y)
    for z0 in range(0, Mz, chunk):
        zz = z[z0:z0 + chunk]
        acc = np.zeros((len(zz), My, Mx))
        for i in range(ngauss):
            gz = np.exp(-(zz - c[i, 2]) ** 2 / (2 * sig[i] ** 2))
            acc += gz[:, None, None] * (gy[i][None, :, None] * gx[i][None, None, :])
        acc += zz[:, None, None] * (cy[None, :, None] * sx[None, None, :])
        out[z0:z0 + len(zz)] = acc
    return out


def paper_2d(M: int = 101) -> np.ndarray:
    """sinc(sqrt(x^2+y^2)) + sinc(2(x-2)^2 + 2(y+2)^2) on [-4,4]^2 (Sec. 3.2.3)."""
    X, Y = mesh([M, M], [-4.0, -4.0], [4.0, 4.0])
    return sinc(np.sqrt(X ** 2 + Y ** 2)) + sinc(2 * (X - 2) ** 2 + 2 * (Y + 2) ** 2)


def paper_3d(M: int = 33) -> np.ndarray:
    """sinc(sqrt(x^2+y^2+z^2)) + sinc(2(x-2)^2 + (y+2)^2 + (z-2)^2) on [-4,4]^3 (Sec. 3.2.3)."""
    X, Y, Z = mesh([M] * 3, [-4.0] * 3, [4.0] * 3)
    return sinc(np.sqrt(X ** 2 + Y ** 2 + Z ** 2)) + sinc(2 * (X - 2) ** 2 + (Y + 2) ** 2 + (Z - 2) ** 2)


def symmetric_sinc_1d(M: int) -> np.ndarray:
    """sinc(x+1) + sinc(x-1) on [-4, 4] (Sec. 3.1.2)."""
    x = axis_coords(M, -4.0, 4.0)
    return sinc(x + 1) + sinc(x - 1)


def asymmetric_sinc_1d(M: int) -> np.ndarray:
    """sinc(x) + sinc(2x-1) + sinc(3x+1.5) on [-4, 4] (Sec. 3.1.1)."""
    x = axis_coords(M, -4.0, 4.0)
    return sinc(x) + sinc(2 * x - 1) + sinc(3 * x + 1.5)


def random_field(npts, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Standard-normal noise on a grid (worst case for conditioning checks)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(tuple(reversed(list(npts)))).astype(dtype)


def tensor_polynomial(npts, degree: int, seed: int = 0) -> np.ndarray:
    """Seeded tensor-product polynomial of per-axis degree <= ``degree`` in the
    unit-box coordinates k/(M_a - 1)."""
    rng = np.random.default_rng(seed)
    d = len(npts)
    coef = rng.standard_normal((d, degree + 1))
    X = mesh(list(npts), [0.0] * d, [1.0] * d)
    out = np.ones_like(X[0])
    for a in range(d):
        out = out * np.polynomial.polynomial.polyval(X[a], coef[a])
    return out


def uniform_points(npts: int, d: int, seed: int = 0) -> np.ndarray:
    """Uniform random points in [0,1]^d, shape (npts, d), for scattered decode."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(npts, d))


def batch_instances(count: int = 4096, seed: int = 0, size2=(32, 512), size3=(16, 128), degrees=(2, 5),
                    cp_ratio: int = 4, dims=(2, 3), dtype=np.float32):
    """Seeded batch of independent grids shaped like the batched-fit workload.

    Instances alternate over ``dims``; per-axis point counts are log-uniform
    in ``size2`` (2-D) or ``size3`` (3-D; 1-D uses ``size2``); the degree is
    uniform in ``degrees``; control points per axis are max(p + 1,
    M // cp_ratio), i.e. nspans = that - p.  Fields alternate between a sum of
    three shifted products of sin(x)/x on [-4 pi, 4 pi]^d and a sum of four
    Gaussians (centres U[0,1]^d, sigma U[0.05, 0.2]) on [0,1]^d.

    Returns (specs, data): specs are dicts with dim, degree, npts, nspans,
    q_offset (grid axis 0 fastest, like a single fit); data is one array.
    """
    rng = np.random.default_rng(seed)
    specs, parts, off = [], [], 0
    for i in range(count):
        d = dims[i % len(dims)]
        lo, hi = size3 if d == 3 else size2
        npts = [int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(d)]
        p = int(rng.integers(degrees[0], degrees[1] + 1))
        nspans = [max(p + 1, M // cp_ratio) - p for M in npts]
        kind = i % 4 < 2
        if kind:
            # sum of shifted separable sinc products on [-4 pi, 4 pi]^d
            xs = [axis_coords(M, -4 * np.pi, 4 * np.pi) for M in npts]
            field = 0.0
            for _ in range(3):
                a = rng.uniform(0.5, 1.0)
                term = None
                for ax in range(d):
                    c = rng.uniform(-2 * np.pi, 2 * np.pi)
                    f = sinc(xs[ax] - c)
                    term = f if term is None else np.multiply.outer(f, term)
                field = field + a * term
        else:
            xs = [axis_coords(M, 0.0, 1.0) for M in npts]
            field = 0.0
            for _ in range(4):
                sig = rng.uniform(0.05, 0.2)
                term = None
                for ax in range(d):
                    c = rng.uniform(0.0, 1.0)
                    f = np.exp(-(xs[ax] - c) ** 2 / (2 * sig * sig))
                    term = f if term is None else np.multiply.outer(f, term)
                field = field + term
        arr = np.asarray(field, dtype=np.float64).astype(dtype).ravel()
        specs.append(dict(dim=d, degree=p, npts=npts, nspans=nspans, q_offset=off))
        parts.append(arr)
        off += arr.size
    return specs, np.concatenate(parts)
