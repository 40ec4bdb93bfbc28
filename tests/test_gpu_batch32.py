"""Batches of independent fits in MFA_PREC_FP32 (FP32 basis, projection and
residual; FP64 factors, solves and control points) against the oracle's
global LSQ fit, instance by instance.

Bar (the mixed form's): decoded RMS within 1 % of the oracle's and max
|decoded difference| <= 1e-5 of the data range.  The 1 % bar holds where the
fit error is far above FP32 rounding of the data, which is the stated rule
for choosing FP32: RMS >= 100 * 2^-24 * range.  Below that rule the FP32 path
is still held to an absolute error of 100 * 2^-24 * range.
"""
import numpy as np
import pytest

from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu

FP32 = mfa.MFA_PREC_FP32
U32 = 2.0 ** -24


def _oracle(spec, data):
    d = spec["dim"]
    npts = spec["npts"]
    Q = data[spec["q_offset"]:spec["q_offset"] + int(np.prod(npts))].astype(np.float64).reshape(tuple(reversed(npts)))
    prob = O.make_problem(spec["degree"], list(npts), list(spec["nspans"]), [1] * d, 0)
    return prob, Q, O.global_fit(prob, Q)


def _check_batch(specs, data, b):
    P = b.ctrl()
    off = b.offsets()
    rms, mx = b.residual(_dev(data))
    D = b.decode(np.empty(data.size, dtype=np.float64))
    for i, sp in enumerate(specs):
        prob, Q, Pref = _oracle(sp, data)
        rng = float(Q.max() - Q.min())
        st = O.residual_stats(prob, Q, Pref)
        Dref = O.decode_grid(prob, Pref).ravel()
        Di = D[sp["q_offset"]:sp["q_offset"] + Dref.size]
        assert np.abs(Di - Dref).max() <= 1e-5 * max(rng, 1e-30), (i, sp)
        if st["rms"] >= 100 * U32 * rng:
            assert abs(rms[i] - st["rms"]) <= 0.01 * st["rms"], (i, rms[i], st["rms"])
        else:
            assert abs(rms[i] - st["rms"]) <= 100 * U32 * rng, (i, rms[i], st["rms"])
        assert abs(mx[i] - np.abs(Q.ravel() - Dref).max()) <= 1e-5 * max(rng, 1e-30)
        # the control points carry the FP32 projection's rounding through the
        # FP64 solves; the decoded values above are the bar, these a sanity check
        Pi = P[off[i]:off[i + 1]]
        assert np.abs(Pi - Pref.ravel()).max() <= 1e-3 * max(np.abs(Pref).max(), 1e-30), (i, sp)
    return rms


def _dev(a):
    import torch
    return torch.from_numpy(a).cuda()


def test_fp32_batch_small_mixed_dims_and_degrees():
    specs, data = inputs.batch_instances(40, seed=21, size2=(14, 90), size3=(10, 30), degrees=(1, 5),
                                         dims=(1, 2, 3))
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, _dev(data), FP32)
        _check_batch(specs, data, b)
        b.free()
    finally:
        h.close()


def test_fp32_batch_large_planes_and_bands():
    """2-D instances large enough to split into bands of y control points,
    and 3-D instances whose xy planes exceed one staging chunk (rows of a
    plane streamed across chunks), beside small ones."""
    rng = np.random.default_rng(5)
    specs, chunks, off = [], [], 0
    shapes = [(2, (300, 260), 3), (2, (512, 200), 5), (2, (101, 517), 2), (3, (128, 96, 12), 3),
              (3, (70, 64, 9), 4), (3, (12, 10, 8), 2), (2, (33, 29), 1), (1, (900,), 3)]
    for d, npts, p in shapes:
        n = int(np.prod(npts))
        x = [np.linspace(-3, 3, m) for m in npts]
        grids = np.meshgrid(*reversed(x), indexing="ij")
        f = np.ones(grids[0].shape)
        for g in grids:
            f = f * np.sinc(g / 2)
        f = f + 0.05 * rng.standard_normal(f.shape)
        chunks.append(f.astype(np.float32).ravel())
        specs.append({"dim": d, "degree": p, "npts": list(npts),
                      "nspans": [max(p + 1, m // 4) - p for m in npts], "q_offset": off})
        off += n
    data = np.concatenate(chunks)
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, _dev(data), FP32)
        _check_batch(specs, data, b)
        b.free()
    finally:
        h.close()


def test_fp32_refit_graph_equals_fresh_encode_and_is_linear():
    specs, data = inputs.batch_instances(30, seed=13, size2=(20, 120), size3=(12, 40), degrees=(2, 5))
    data2 = (2.0 * data).astype(np.float32)  # a power-of-two scale commutes with every rounding
    h = mfa.Handle(0)
    try:
        q1, q2 = _dev(data), _dev(data2)
        b = h.encode_batch(specs, q1, FP32)
        b.refit(q2)
        b.refit(q2)  # replay
        P2 = b.ctrl()
        # autotuned: CTA item size for the batch, solve block size per group
        for g in b.group_tuning():
            assert g["item_pts"] in (16384, 32768, 131072)
            assert min(g["candidate_ms"][:6]) > 0
            assert g["chosen_ms"] == min(g["candidate_ms"][:3])
            assert g["candidate_ms"][(32, 64, 128).index(g["tile_s"])] == g["chosen_ms"]
            k = (16384, 32768, 131072).index(g["item_pts"])
            assert g["candidate_ms"][3 + k] == min(g["candidate_ms"][3:6])
        c = h.encode_batch(specs, q2, FP32)
        assert np.array_equal(P2, c.ctrl())
        b.refit(q1)
        P1 = b.ctrl()
        assert np.array_equal(P2, 2.0 * P1)
        # scattered decode of the FP32 batch's FP64 control points
        rng = np.random.default_rng(0)
        pts = rng.uniform(0, 1, (len(specs) * 16, 3))
        qinst = np.arange(len(specs), dtype=np.int32)
        pt_off = np.arange(0, len(pts) + 1, 16, dtype=np.int64)
        vals = b.decode_points(qinst, pt_off, pts)
        off = b.offsets()
        for i, sp in enumerate(specs[:6]):
            prob = O.make_problem(sp["degree"], list(sp["npts"]), list(sp["nspans"]), [1] * sp["dim"], 0)
            Pi = P1[off[i]:off[i + 1]].reshape(tuple(reversed([s + sp["degree"] for s in sp["nspans"]])))
            want = O.scattered_decode(prob, Pi, pts[16 * i:16 * i + 16, :sp["dim"]])
            assert np.abs(vals[16 * i:16 * i + 16] - want).max() <= 1e-9 * max(1.0, np.abs(want).max())
        b.free()
        c.free()
    finally:
        h.close()


def test_fp32_host_data_residual_on_the_staged_copy():
    specs, data = inputs.batch_instances(16, seed=4, size2=(20, 80), size3=(12, 30), degrees=(2, 4))
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, data, FP32)
        rms, mx = b.residual()
        rms2, mx2 = b.residual(_dev(data))
        assert np.array_equal(rms, rms2) and np.array_equal(mx, mx2)
        b.free()
    finally:
        h.close()


def test_fp32_batch_refuses_what_it_does_not_cover():
    specs, data = inputs.batch_instances(4, seed=1, size2=(20, 40), size3=(12, 20), degrees=(2, 3))
    h = mfa.Handle(0)
    try:
        with pytest.raises(mfa.MFAError) as e:
            h.encode_batch(specs, _dev(data.astype(np.float64)), FP32)
        assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
        big = [{"dim": 2, "degree": 3, "npts": [5000, 8], "nspans": [1200, 4], "q_offset": 0}]
        with pytest.raises(mfa.MFAError) as e:
            h.encode_batch(big, _dev(np.zeros(40000, np.float32)), FP32)
        assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    finally:
        h.close()


def _grid_field(npts, rng):
    x = [np.linspace(-3, 3, m) for m in npts]
    grids = np.meshgrid(*reversed(x), indexing="ij")
    f = np.ones(grids[0].shape)
    for g in grids:
        f = f * np.sinc(g / 2)
    return (f + 0.05 * rng.standard_normal(f.shape)).astype(np.float32).ravel()


def test_fp32_batch_edge_shapes():
    """Degrees 1, 6 and 7; the longest row the staging takes (1023 points);
    256 x control points (eight column groups of open y control points);
    single-span axes; interpolation (as many points as control points);
    small 3-D planes several to a chunk; a 2-D instance whose y spans split
    over warps with the fewest spans per warp (p); a 3-D instance with 100 x
    50 control points per plane (its z-expanded planes larger than a warp's
    share of shared memory)."""
    rng = np.random.default_rng(8)
    shapes = [
        (1, (1023,), 3, None), (2, (1023, 9), 4, None), (2, (1023, 12), 2, [253, 3]),
        (1, (60,), 1, None), (2, (40, 37), 6, None), (3, (30, 28, 26), 7, None),
        (2, (16, 16), 5, [1, 1]), (3, (12, 10, 40), 2, None), (2, (9, 9), 3, [6, 6]),
        (2, (200, 300), 5, [5 * 8, 5 * 8]), (1, (7,), 6, [1]), (3, (400, 200, 6), 3, None),
    ]
    specs, chunks, off = [], [], 0
    for d, npts, p, ns in shapes:
        n = int(np.prod(npts))
        chunks.append(_grid_field(npts, rng))
        nspans = ns if ns is not None else [max(p + 1, m // 4) - p for m in npts]
        specs.append({"dim": d, "degree": p, "npts": list(npts), "nspans": list(nspans), "q_offset": off})
        off += n
    data = np.concatenate(chunks)
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, _dev(data), FP32)
        _check_batch(specs, data, b)
        b.refit(_dev(data))  # autotune + captured graph on the same shapes
        _check_batch(specs, data, b)
        b.free()
    finally:
        h.close()


def test_fp32_unit_pipeline_equals_the_pass_by_pass_fit():
    """The fit as one pipeline per (class, degree) unit on side streams (the
    untraced path) gives the same control points, bit for bit, as the fit
    run pass by pass (the traced path), refined and unrefined instances of
    every degree and of both classes included."""
    specs, data = inputs.batch_instances(48, seed=17, size2=(20, 120), size3=(12, 40), degrees=(1, 5),
                                         dims=(1, 2, 3))
    h = mfa.Handle(0)
    try:
        b1 = h.encode_batch(specs, _dev(data), FP32)
        P1 = b1.ctrl()
        mfa.mfa_trace_enable(h.h, True)
        b2 = h.encode_batch(specs, _dev(data), FP32)
        mfa.mfa_trace_enable(h.h, False)
        P2 = b2.ctrl()
        assert b1.info()["refined"] > 0
        assert np.array_equal(P1, P2)
        b1.free()
        b2.free()
    finally:
        h.close()
