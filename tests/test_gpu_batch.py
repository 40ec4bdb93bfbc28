"""Batches of independent fits (one subdomain each) against the oracle's
global LSQ fit (Eq. minimization-problem, N = 1), instance by instance."""
import numpy as np
import pytest

from mfa_cases import TOL_FP64, rel_diff
from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu


def _oracle(spec, data):
    d = spec["dim"]
    npts = spec["npts"]
    Q = data[spec["q_offset"]:spec["q_offset"] + int(np.prod(npts))].astype(np.float64).reshape(tuple(reversed(npts)))
    prob = O.make_problem(spec["degree"], list(npts), list(spec["nspans"]), [1] * d, 0)
    P = O.global_fit(prob, Q)
    return prob, Q, P


def _small_batch(seed, count=30):
    return inputs.batch_instances(count, seed=seed, size2=(14, 70), size3=(10, 26), degrees=(1, 5), dims=(1, 2, 3))


@pytest.mark.parametrize("precision", [mfa.MFA_PREC_FP64, mfa.MFA_PREC_MIXED])
def test_batch_matches_oracle_per_instance(precision):
    import torch
    specs, data = _small_batch(7)
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, torch.from_numpy(data).cuda(), precision)
        P = b.ctrl()
        off = b.offsets()
        rms, mx = b.residual(torch.from_numpy(data).cuda())
        D = b.decode(np.empty(data.size, dtype=np.float64))
        for i, sp in enumerate(specs):
            prob, Q, Pref = _oracle(sp, data)
            Pi = P[off[i]:off[i + 1]]
            assert rel_diff(Pi, Pref.ravel()) <= TOL_FP64, (i, sp)
            st = O.residual_stats(prob, Q, Pref)
            assert abs(rms[i] - st["rms"]) <= 0.01 * st["rms"] + 1e-15, (i, rms[i], st["rms"])
            Dref = O.decode_grid(prob, Pref).ravel()
            Di = D[sp["q_offset"]:sp["q_offset"] + Dref.size]
            rng = float(Q.max() - Q.min())
            assert np.abs(Di - Dref).max() <= 1e-9 * max(rng, 1.0)
            assert abs(mx[i] - np.abs(Q.ravel() - Dref).max()) <= 1e-5 * max(rng, 1.0)
        b.free()
    finally:
        h.close()


def test_batch_refit_graph_equals_fresh_encode():
    """The captured refit on new data gives the same control points as a
    fresh batch encode of that data; replays on the same pointer reuse it."""
    import torch
    specs, data = _small_batch(11, count=20)
    data2 = (2.0 * data).astype(np.float32)  # exact: a power-of-two scale commutes with every rounding
    h = mfa.Handle(0)
    try:
        q1 = torch.from_numpy(data).cuda()
        q2 = torch.from_numpy(data2).cuda()
        b = h.encode_batch(specs, q1, mfa.MFA_PREC_MIXED)
        rc0, sizes0, _ = b.tile_sizes()
        assert rc0 == mfa.MFA_NOT_CONVERGED and sizes0 == [128, 64, 256]
        b.refit(q2)
        rc1, sizes1, cand = b.tile_sizes()  # tuned by timing on the first refit
        assert rc1 == mfa.MFA_OK and sizes1[0] in (64, 128, 256) and sizes1[1] in (32, 64, 128)
        assert (cand > 0).all()
        # every (dimension, degree) group keeps its own fastest candidate
        for g in b.group_tuning():
            tiled = g["candidate_ms"][:9]
            assert min(tiled) > 0
            opts = tiled + ([g["candidate_ms"][9]] if g["candidate_ms"][9] >= 0 else [])
            assert g["chosen_ms"] == min(opts)
            if not g["fused"]:
                k = 3 * (64, 128, 256).index(g["tile_c"]) + (32, 64, 128).index(g["tile_s"])
                assert tiled[k] == g["chosen_ms"]
            else:
                assert g["dim"] == 3 and g["candidate_ms"][9] == g["chosen_ms"]
        b.refit(q2)  # replay of the captured graph
        P2 = b.ctrl()
        b.refit(q2)
        assert np.array_equal(P2, b.ctrl())
        # a fresh encode takes the default path per group (the fused 3-D path
        # sums in another order): equal to the FP64 bar
        c = h.encode_batch(specs, q2, mfa.MFA_PREC_MIXED)
        assert rel_diff(P2, c.ctrl()) <= TOL_FP64
        b.refit(q1)  # new pointer: captured again
        P1 = b.ctrl()
        d = h.encode_batch(specs, q1, mfa.MFA_PREC_MIXED)
        assert rel_diff(P1, d.ctrl()) <= TOL_FP64
        # linearity, exactly: fit(2 q) = 2 fit(q) bit for bit
        assert np.array_equal(P2, 2.0 * P1)
        for x in (b, c, d):
            x.free()
    finally:
        h.close()


def test_batch_host_data_and_staged_residual():
    specs, data = _small_batch(3, count=12)
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, data, mfa.MFA_PREC_FP64)
        r1, m1 = b.residual(None)
        r2, m2 = b.residual(data)
        assert np.array_equal(r1, r2) and np.array_equal(m1, m2)
        b.free()
    finally:
        h.close()


def test_batch_layout_rejection():
    """An instance with more control points than data points along an axis
    fails the Schoenberg-Whitney precheck: no batch is created."""
    specs, data = _small_batch(5, count=4)
    bad = dict(specs[1])
    bad["nspans"] = [bad["npts"][0] + 3] + list(bad["nspans"][1:])
    specs[1] = bad
    h = mfa.Handle(0)
    try:
        with pytest.raises(mfa.MFAError) as ei:
            h.encode_batch(specs, data, mfa.MFA_PREC_MIXED)
        assert ei.value.code == mfa.MFA_ERR_LAYOUT
    finally:
        h.close()


def test_batch_decode_points_matches_grid_and_oracle():
    """Scattered decode of batch instances: at the grid parameters it equals
    the batch's grid decode; at random parameters it equals the oracle's
    decode of the oracle fit."""
    import torch
    specs, data = _small_batch(13, count=10)
    h = mfa.Handle(0)
    rng = np.random.default_rng(0)
    try:
        b = h.encode_batch(specs, torch.from_numpy(data).cuda(), mfa.MFA_PREC_FP64)
        D = b.decode(np.empty(data.size, dtype=np.float64))
        qinst, off, pts, ref = [], [0], [], []
        for i, sp in enumerate(specs):
            d, npts = sp["dim"], sp["npts"]
            grids = [np.arange(M) / max(M - 1, 1) for M in npts]
            mesh = np.stack(np.meshgrid(*reversed(grids), indexing="ij"), -1).reshape(-1, d)[:, ::-1]
            P3 = np.zeros((len(mesh), 3))
            P3[:, :d] = mesh
            qinst.append(i)
            pts.append(P3)
            off.append(off[-1] + len(P3))
            ref.append(D[sp["q_offset"]:sp["q_offset"] + len(P3)])
        vals = b.decode_points(qinst, off, np.concatenate(pts))
        assert np.abs(vals - np.concatenate(ref)).max() <= 1e-11 * max(1.0, np.abs(data).max())
        # random parameters against the oracle
        for i in (0, 4, 7):
            sp = specs[i]
            prob, Q, Pref = _oracle(sp, data)
            u = rng.uniform(0, 1, size=(257, 3))
            got = b.decode_points([i], [0, len(u)], u)
            want = O.scattered_decode(prob, Pref, u[:, :sp["dim"]])
            assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max())
        b.free()
    finally:
        h.close()


@pytest.mark.parametrize("degrees", [(1, 5), (1, 1), (2, 2), (3, 3), (4, 4), (6, 7)])
def test_batch_decode_points_float_float(degrees):
    """Scattered decode of a mixed-precision batch (float-float control
    points, float-float arithmetic): equal to the oracle's decode of the
    batch's own control points at random parameters, at the knots, at 0 and
    1, and at parameters outside [0, 1] (clamped).  One degree per batch runs
    the kernel compiled for that degree; several degrees, the general one."""
    import torch
    specs, data = inputs.batch_instances(12, seed=21, size2=(14, 70), size3=(10, 26), degrees=degrees,
                                         dims=(1, 2, 3))
    h = mfa.Handle(0)
    rng = np.random.default_rng(3)
    try:
        b = h.encode_batch(specs, torch.from_numpy(data).cuda(), mfa.MFA_PREC_MIXED)
        P = b.ctrl()
        off = b.offsets()
        qinst, poff, pts, want = [], [0], [], []
        for i, sp in enumerate(specs):
            d, p = sp["dim"], sp["degree"]
            ncp = [n + p for n in sp["nspans"]]
            prob = O.make_problem(p, list(sp["npts"]), list(sp["nspans"]), [1] * d, 0)
            Pi = P[off[i]:off[i + 1]].reshape(tuple(reversed(ncp)))
            u = rng.uniform(0, 1, size=(200, 3))
            ns = max(sp["nspans"])
            knots = np.arange(ns + 1) / ns
            u[:len(knots), 0] = knots
            u[len(knots):len(knots) + 4] = [[0, 0, 0], [1, 1, 1], [-0.25, 1.5, 0.5], [1.75, -1e-3, 1.0]]
            qinst.append(i)
            pts.append(u)
            poff.append(poff[-1] + len(u))
            want.append(O.scattered_decode(prob, Pi, np.clip(u[:, :d], 0.0, 1.0)))
        got = b.decode_points(qinst, poff, np.concatenate(pts))
        for i in range(len(specs)):
            g = got[poff[i]:poff[i + 1]]
            scale = max(1.0, np.abs(P[off[i]:off[i + 1]]).max())
            assert np.abs(g - want[i]).max() <= 1e-12 * scale, (i, specs[i])
        b.free()
    finally:
        h.close()


def test_batch_of_many_small_3d_fits_fused_path():
    """Many similar small 3-D fits (no instance dominates the batch): the
    fused float-float kernels run one CTA per instance; every instance checked
    matches the oracle within 1e-9 and the RMS within 1 %."""
    import torch
    rng = np.random.default_rng(4)
    specs, parts, off = [], [], 0
    for i in range(400):
        npts = [int(rng.integers(11, 15)), int(rng.integers(10, 14)), int(rng.integers(9, 13))]
        nsp = [max(1, M // 4 - 3 + 1) for M in npts]
        Q = inputs.gauss_3d(tuple(npts), seed=100 + i, ngauss=3, dtype=np.float32)
        specs.append(dict(dim=3, degree=3, npts=npts, nspans=nsp, q_offset=off))
        parts.append(Q.ravel())
        off += Q.size
    data = np.concatenate(parts)
    h = mfa.Handle(0)
    try:
        b = h.encode_batch(specs, torch.from_numpy(data).cuda(), mfa.MFA_PREC_MIXED)
        P = b.ctrl()
        offs = b.offsets()
        rms, _ = b.residual(torch.from_numpy(data).cuda())
        for i in range(0, 400, 37):
            prob, Q, Pref = _oracle(specs[i], data)
            assert rel_diff(P[offs[i]:offs[i + 1]], Pref.ravel()) <= TOL_FP64, i
            st = O.residual_stats(prob, Q, Pref)
            assert abs(rms[i] - st["rms"]) <= 0.01 * st["rms"] + 1e-15
        b.free()
    finally:
        h.close()
