"""Which stages of the fit need more than FP32 (test infrastructure, CPU only).

Global tensor-product LSQ fit (N = 1) of the 3-D Gaussian-sum field at a given
size, computed separably as in the oracle (project every axis with N^T, then
solve the per-axis normal equations, Eq. minimization-problem), once in FP64
and then with one stage at a time replaced by its FP32 counterpart:

  A  first projection axis in FP32 (products and sums)
  A2 first projection axis with the basis rounded to FP32, exact arithmetic
  B  every projection axis in FP32
  C  the normal-equation solves in FP32 (Cholesky factors and triangular solves)
  D  the decode of the FP64 fit in FP32
  F  everything in FP32 (residual formed in FP64)

Each line reports the decoded RMS error, its change against the FP64 fit, the
max error and the relative control-point difference.  The 1 % RMS bar of the
mixed-precision path fails for every FP32 stage at 512^3 (192 spans, p = 3),
because the fit error of that workload sits at the FP32 rounding level of its
O(1) data.

Usage: python oracle/precision_study.py [M] [nspans]   (512 192: ~5 min, ~20 GB)
"""
import os
import sys

import numpy as np
import scipy.linalg as sl

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import mfa_oracle as O  # noqa: E402
from paper_2210_06528_gb300 import inputs  # noqa: E402


def main(M=512, nspans=192, p=3):
    Q32 = inputs.gauss_3d((M, M, M), seed=0)
    Q = Q32.astype(np.float64)
    N = O.basis_matrix(O.clamped_uniform_knots(nspans, p), p, O.grid_params(M))
    N32 = N.astype(np.float32)
    A = N.T @ N

    def project(T, mats, dt):
        for a in range(3):
            T = O.apply_along_axis(T, mats[a].T.astype(dt), a)
        return T

    def solve(B, fp32=False):
        if not fp32:
            Ainv = np.linalg.solve(A, np.eye(A.shape[0]))
            for a in range(3):
                B = O.apply_along_axis(B, Ainv, a)
            return B
        Lc = np.linalg.cholesky(A).astype(np.float32)
        for a in range(3):
            ax = O._np_axis(a, 3)
            Bm = np.moveaxis(B.astype(np.float32), ax, 0)
            sh = Bm.shape
            Y = sl.solve_triangular(Lc, Bm.reshape(sh[0], -1), lower=True)
            X = sl.solve_triangular(Lc.T, Y, lower=False)
            B = np.moveaxis(X.reshape(sh), 0, ax)
        return B.astype(np.float64)

    def rms(P):
        E = Q - O.decode_box(np.asarray(P, np.float64), [N] * 3)
        return np.sqrt(np.mean(E * E)), np.abs(E).max()

    P64 = solve(project(Q, [N] * 3, np.float64))
    r0, m0 = rms(P64)
    print(f"FP64 fit: rms {r0:.6e}  max {m0:.3e}")

    def report(name, P):
        r, m = rms(P)
        dP = np.abs(P - P64).max() / np.abs(P64).max()
        print(f"{name:44s} rms {r:.6e} ({100 * (r / r0 - 1):+8.3f}%)  max {m:.3e}  dP {dP:.2e}")

    T = O.apply_along_axis(Q32, N32.T, 0).astype(np.float64)
    report("A  first projection axis FP32", solve(project_rest(T, N)))
    T = O.apply_along_axis(Q, N32.astype(np.float64).T, 0)
    report("A2 first axis, basis rounded to FP32", solve(project_rest(T, N)))
    report("B  every projection axis FP32", solve(project(Q32, [N32] * 3, np.float32).astype(np.float64)))
    report("C  normal-equation solves FP32", solve(project(Q, [N] * 3, np.float64), fp32=True))
    E = Q - O.decode_box(P64.astype(np.float32), [N32] * 3).astype(np.float64)
    r = np.sqrt(np.mean(E * E))
    print(f"{'D  decode FP32 (FP64 fit)':44s} rms {r:.6e} ({100 * (r / r0 - 1):+8.3f}%)  max {np.abs(E).max():.3e}")
    report("F  everything FP32", solve(project(Q32, [N32] * 3, np.float32), fp32=True))


def project_rest(T, N):
    """Axes 1 and 2 of the projection in FP64."""
    return O.apply_along_axis(O.apply_along_axis(T, N.T, 1), N.T, 2)


if __name__ == "__main__":
    a = [int(x) for x in sys.argv[1:3]]
    main(*a)
