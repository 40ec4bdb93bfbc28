"""Full-size and workload-shaped parity of the mixed-precision path.

Mixed path bar: decoded RMS error within 1% of the oracle's and
max |decoded difference| <= 1e-5 of the data range.  The mixed path uses
float-float sums on the FP32 pipes, so its control points are also held to
the FP64 bar (relative difference <= 1e-9).
"""
import numpy as np
import pytest

from mfa_cases import TOL_FP64, GpuFit, oracle_problem, rel_diff
from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu


def _mixed_case(Q, p, nspans, nsub, delta, tol, max_iters=50, check_decode=True):
    Qd = Q.astype(np.float64)
    prob = oracle_problem(Qd, p, nspans, nsub, delta)
    ref = O.schwarz_solve(prob, Qd, max_iters=max_iters, tol_dP=tol)
    g = GpuFit(Q, p, nspans, nsub, delta, precision=mfa.MFA_PREC_MIXED)
    try:
        rc, rep = g.iterate(max_iters, tol)
        assert rep.iters == ref["iters"]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
        res = g.residual()
        oref = O.residual_stats(prob, Qd, ref["P"])
        assert abs(res.rms_decoded - oref["rms"]) <= 0.01 * oref["rms"], (res.rms_decoded, oref["rms"])
        rng = float(Qd.max() - Qd.min())
        if check_decode:
            D = g.decode_grid(np.float64)
            Dref = O.decode_grid(prob, ref["P"])
            assert np.abs(D - Dref).max() <= 1e-5 * rng
        return res, oref
    finally:
        g.close()


def test_mixed_3d_workload_shape_128():
    """128^3 sample with the 512^3 workload's per-subdomain shape (p=3,
    24-span cores, overlap 2, 2.67 points per span), stop at dP_rel <= 1e-7."""
    Q = inputs.gauss_3d((128, 128, 128), seed=0, dtype=np.float32)
    _mixed_case(Q, 3, [48, 48, 48], [2, 2, 2], 2, 1e-7)


def test_mixed_2d_ragged_uneven():
    Q = inputs.sinc_2d(300, noise=1e-3, seed=4, dtype=np.float32)
    _mixed_case(Q, 3, [70, 61], [3, 2], 2, 1e-9)


@pytest.mark.slow
def test_fullsize_3d_512_mixed():
    """The bench workload itself: 512^3, 8x8x8 subdomains of 24 core spans,
    p = 3, overlap 2, mixed precision, stop at dP_rel <= 1e-7 (full oracle run)."""
    Q = inputs.gauss_3d((512, 512, 512), seed=0, dtype=np.float32)
    _mixed_case(Q, 3, [192] * 3, [8] * 3, 2, 1e-7, check_decode=False)


@pytest.mark.slow
def test_fullsize_2d_1024_mixed():
    """2-D workload: 1024^2 sinc(x)sinc(y) + N(0,1e-3), 4x4 subdomains of 64 core spans."""
    Q = inputs.sinc_2d(1024, noise=1e-3, seed=0, dtype=np.float32)
    _mixed_case(Q, 3, [256, 256], [4, 4], 2, 1e-6)


@pytest.mark.parametrize("p,delta,nsub,nspans,npts", [
    (2, 1, (2, 3, 2), (14, 16, 12), (41, 47, 35)),
    (3, 0, (2, 2, 2), (12, 12, 12), (37, 33, 35)),
    (4, 3, (2, 2, 1), (12, 10, 8), (45, 40, 31)),
    (5, 2, (2, 1, 2), (14, 8, 12), (50, 33, 46)),
    (3, 6, (3, 2, 2), (15, 12, 12), (43, 38, 37)),
])
def test_mixed_3d_degrees_and_overlaps(p, delta, nsub, nspans, npts):
    """Mixed path in 3-D (fused projection) across degrees, overlaps, ragged
    grids and uneven splits: control points within 1e-9 of the oracle."""
    Q = inputs.gauss_3d(npts, seed=p, dtype=np.float32)
    _mixed_case(Q, p, list(nspans), list(nsub), delta, 1e-9, max_iters=60)


@pytest.mark.parametrize("p,delta,nsub,nspans,npts", [
    (2, 2, (2, 2, 2), (16, 14, 12), (48, 41, 39)),
    (4, 2, (2, 2, 1), (14, 12, 10), (56, 47, 43)),
    (5, 3, (2, 1, 2), (14, 10, 12), (64, 45, 50)),
])
def test_mixed_3d_degrees_row_aligned(p, delta, nsub, nspans, npts):
    """Rows a multiple of 16 bytes long on an aligned base: the projection
    stages the data with tensor copies; control points within 1e-9 of the
    oracle across degrees."""
    Q = inputs.gauss_3d(npts, seed=10 + p, dtype=np.float32)
    _mixed_case(Q, p, list(nspans), list(nsub), delta, 1e-9, max_iters=60)


def test_mixed_3d_unaligned_base_matches_aligned():
    """The same data on a device base that is not 16-byte aligned is staged
    element by element; the fit is bit-identical to the tensor-copy staging."""
    import torch
    Q = inputs.gauss_3d((64, 56, 48), seed=11, dtype=np.float32)
    a = GpuFit(Q, 3, [20, 18, 16], [2, 2, 2], 2, precision=mfa.MFA_PREC_MIXED)
    h = mfa.Handle(0)
    try:
        a.iterate(4, 0.0)
        Pa = a.ctrl()
        buf = torch.empty(Q.size + 1, dtype=torch.float32, device="cuda")
        buf[1:] = torch.from_numpy(Q.ravel()).cuda()
        qd = buf[1:].view(Q.shape)
        assert qd.data_ptr() % 16 != 0
        m = h.encode(qd, a.layout)
        m.iterate(4, 0.0)
        Pb = m.ctrl()
        m.free()
        assert np.array_equal(Pa, Pb)
    finally:
        a.close()
        h.close()
