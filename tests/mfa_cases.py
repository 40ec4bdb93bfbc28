"""Shared helpers for the GPU parity tests: run the CUDA library through its
C ABI and the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import mfa

# FP64 path: relative control-point difference (max |dP| / max |P|)
TOL_FP64 = 1e-9


def layout_for(Q, p, nspans, nsub, delta, precision, cores=None, lo=None, hi=None, knots=mfa.MFA_KNOTS_FLOATING,
               weights=None):
    npts = list(reversed(Q.shape))
    d = len(npts)
    if np.isscalar(delta):
        delta = [delta] * d
    return mfa.make_layout(d, p, npts, nspans, nsub, delta, precision, core_spans=cores, lo=lo, hi=hi, knots=knots,
                           weights=weights)


def oracle_problem(Q, p, nspans, nsub, delta, cores=None, clamped=False, weights=None):
    npts = list(reversed(Q.shape))
    return O.make_problem(p, npts, list(nspans), list(nsub), delta, cores=cores, clamped=clamped, weights=weights)


def rel_diff(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


class GpuFit:
    """One model on the GPU; keeps the handle alive."""

    def __init__(self, Q, p, nspans, nsub, delta, precision=mfa.MFA_PREC_FP64, cores=None, on_device=True,
                 lo=None, hi=None, knots=mfa.MFA_KNOTS_FLOATING, weights=None):
        import torch
        self.handle = mfa.Handle(0)
        self.layout = layout_for(Q, p, nspans, nsub, delta, precision, cores, lo, hi, knots, weights)
        self.q = torch.from_numpy(np.ascontiguousarray(Q)).cuda() if on_device else np.ascontiguousarray(Q)
        self.model = self.handle.encode(self.q, self.layout)

    def ctrl(self):
        return self.model.ctrl()

    def iterate(self, n, tol=0.0, tol_rms_stall=0.0):
        return self.model.iterate(n, tol, tol_rms_stall)

    def residual(self):
        return self.model.residual(self.q)

    def decode_grid(self, dtype=np.float64):
        out = np.empty(self.q.shape, dtype=dtype)
        self.model.decode_grid(out)
        return out

    def close(self):
        self.model.free()
        self.handle.close()
