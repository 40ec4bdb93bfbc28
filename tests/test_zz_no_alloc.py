"""The grid decode that allocates nothing, against the allocating decode.

Some callers cannot allocate device memory at the moment they decode: a
plugin running inside an application that already owns the whole device
through its own memory pool, or a loop that must not stall on cudaMalloc /
cudaFree (both may synchronise the device).  mfa_decode_grid_noalloc serves
them: the caller passes the control points and the output buffer, and every
intermediate lives in one fixed static device array.  Here it must give the
same values as mfa_decode on two calls in a row (with different shapes, so
the second call runs on the first call's leftover scratch contents).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from mfa_cases import GpuFit, oracle_problem
from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu

# same bound as the decode comparisons of the parity tests
TOL = 1e-10


def _reference(Q, p, nspans, nsub, delta):
    import torch
    g = GpuFit(Q, p, nspans, nsub, delta)
    g.iterate(2)
    ref = torch.empty(Q.shape, dtype=torch.float64, device="cuda")
    g.model.decode_grid(ref)  # the allocating entry point
    Ph = np.ascontiguousarray(g.ctrl())
    P = torch.from_numpy(Ph).cuda()
    torch.cuda.synchronize()
    g.close()
    # and the oracle's decode of the same control points
    oref = O.decode_grid(oracle_problem(Q, p, nspans, nsub, delta), Ph)
    return ref, P, oref


def test_noalloc_decode_matches_decode_on_consecutive_calls():
    import torch
    cases = [
        (inputs.paper_2d(97), 3, [30, 27], [2, 3], 1),
        (inputs.paper_3d(29), 2, [12, 11, 10], [2, 2, 2], 1),
        (inputs.asymmetric_sinc_1d(301), 4, [60], [3], 2),
    ]
    stream = torch.cuda.current_stream().cuda_stream
    for Q, p, nspans, nsub, delta in cases:
        ref, P, oref = _reference(Q, p, nspans, nsub, delta)
        npts = list(reversed(Q.shape))
        for call in range(2):
            out = torch.full(Q.shape, float("nan"), dtype=torch.float64, device="cuda")
            mfa.mfa_decode_grid_noalloc(len(npts), p, npts, nspans, P.data_ptr(), out.data_ptr(), stream)
            torch.cuda.synchronize()
            err = (out - ref).abs().max().item()
            assert err <= TOL * max(ref.abs().max().item(), 1.0), (Q.shape, call, err)
            err_o = np.abs(out.cpu().numpy() - oref).max()
            assert err_o <= TOL * max(np.abs(oref).max(), 1.0), (Q.shape, call, err_o)


def test_noalloc_decode_rejects_requests_beyond_its_scratch():
    import torch
    P = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 2-D 8192 x 4096 from 1024 x 1024 spans: the intermediate alone is 8192 * 1027 doubles > 32 MiB
    with pytest.raises(mfa.MFAError) as e:
        mfa.mfa_decode_grid_noalloc(2, 3, [8192, 4096], [1024, 1024], P.data_ptr(), out.data_ptr(), 0)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    with pytest.raises(mfa.MFAError) as e:
        mfa.mfa_decode_grid_noalloc(2, 0, [10, 10], [3, 3], P.data_ptr(), out.data_ptr(), 0)
    assert e.value.code == mfa.MFA_ERR_ARG
