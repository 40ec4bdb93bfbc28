"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

FP64 path: every iterate's control points agree with the oracle's to a
relative difference <= 1e-9 (max |dP| / max |P|).
Mixed path: decoded RMS within 1% of the oracle's and max |decoded difference|
<= 1e-5 of the data range.
"""
import numpy as np
import pytest

from mfa_cases import TOL_FP64, GpuFit, oracle_problem, rel_diff
from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu


def _iterate_parity(Q, p, nspans, nsub, delta, iters, cores=None, on_device=True, update="average"):
    prob = oracle_problem(Q, p, nspans, nsub, delta, cores)
    g = GpuFit(Q, p, nspans, nsub, delta, cores=cores, on_device=on_device)
    try:
        if update == "owner":
            g.model.set_update_rule(mfa.MFA_UPDATE_OWNER)
        st = O.schwarz_initial(prob, Q, update)
        assert rel_diff(g.ctrl(), st.P) <= TOL_FP64, "iteration 0"
        for k in range(1, iters + 1):
            st = O.schwarz_step(prob, Q, st, update)
            rc, rep = g.iterate(1)
            assert rep.iters == k
            assert rel_diff(g.ctrl(), st.P) <= TOL_FP64, f"iteration {k}"
            h = st.history[-1]
            assert abs(rep.dP_rel - h["dP_rel"]) <= 1e-11 + 1e-6 * h["dP_rel"]
            assert abs(rep.jump_max - h["spread"]) <= 1e-11 * max(np.abs(st.P).max(), 1) + 1e-6 * h["spread"]
        res = g.residual()
        ref = O.residual_stats(prob, Q, st.P)
        assert abs(res.rms_decoded - ref["rms"]) <= 1e-8 * max(ref["rms"], 1e-12) + 1e-13
        assert abs(res.maxabs_decoded - ref["max"]) <= 1e-8 * max(ref["max"], 1e-12) + 1e-13
        assert abs(res.data_range - (Q.max() - Q.min())) <= 1e-12 * (Q.max() - Q.min())
        D = g.decode_grid()
        Dref = O.decode_grid(prob, st.P)
        assert np.abs(D - Dref).max() <= 1e-10 * max(np.abs(Dref).max(), 1)
    finally:
        g.close()


def test_config1_sinc_1d_fp64_full():
    """1-D plain method: 1024 points of sin(x)/x on [-4pi, 4pi], p=3, 4 subdomains
    of 32 core spans, overlap 2, Schwarz to dP_rel <= 1e-10."""
    Q = inputs.sinc_1d(1024)
    prob = oracle_problem(Q, 3, [128], [4], 2)
    ref = O.schwarz_solve(prob, Q, max_iters=200, tol_dP=1e-10, keep_iterates=True)
    g = GpuFit(Q, 3, [128], [4], 2)
    try:
        assert rel_diff(g.ctrl(), ref["iterates"][0]) <= TOL_FP64
        rc, rep = g.iterate(200, 1e-10)
        assert rc == mfa.MFA_OK
        assert rep.iters == ref["iters"]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
        res = g.residual()
        oref = O.residual_stats(prob, Q, ref["P"])
        assert abs(res.rms_decoded - oref["rms"]) <= 1e-6 * oref["rms"]
    finally:
        g.close()


@pytest.mark.parametrize("p,delta", [(1, 0), (1, 1), (2, 1), (3, 0), (3, 2), (3, 3), (4, 2), (5, 1), (5, 6)])
def test_1d_iterates(p, delta):
    M = 301  # ragged: 301 points over 60 spans
    Q = inputs.asymmetric_sinc_1d(M)
    _iterate_parity(Q, p, [60], [4], delta, iters=4)


def test_1d_uneven_cores_and_host_input():
    Q = inputs.symmetric_sinc_1d(257)
    _iterate_parity(Q, 3, [50], [4], 2, iters=3, cores=[[9, 17, 4, 20]], on_device=False)


@pytest.mark.parametrize("p,delta,nsub", [(2, 1, (3, 2)), (3, 2, (2, 3)), (3, 0, (4, 4)), (3, 3, (3, 3)),
                                          (4, 4, (2, 2))])
def test_2d_iterates(p, delta, nsub):
    Q = inputs.paper_2d(97)  # 97 x 97 grid (ragged against the spans)
    _iterate_parity(Q, p, [30, 27], list(nsub), delta, iters=3)


def test_2d_rectangular_noise():
    Q = inputs.random_field((83, 61), seed=11)
    _iterate_parity(Q, 2, [26, 18], [3, 2], 1, iters=3)


@pytest.mark.parametrize("p,delta,nsub", [(2, 1, (2, 2, 2)), (3, 2, (3, 2, 2)), (3, 0, (2, 2, 2)),
                                          (3, 3, (2, 2, 2))])
def test_3d_iterates(p, delta, nsub):
    Q = inputs.paper_3d(29)
    _iterate_parity(Q, p, [12, 11, 10], list(nsub), delta, iters=2)


def test_3d_anisotropic_fp32_input():
    Q = inputs.gauss_3d((37, 29, 23), seed=3, dtype=np.float32)
    Qd = Q.astype(np.float64)
    prob = oracle_problem(Qd, 3, [12, 9, 7], [2, 2, 1], 2)
    g = GpuFit(Q, 3, [12, 9, 7], [2, 2, 1], 2)
    try:
        st = O.schwarz_initial(prob, Qd)
        assert rel_diff(g.ctrl(), st.P) <= TOL_FP64
        for _ in range(3):
            st = O.schwarz_step(prob, Qd, st)
            g.iterate(1)
            assert rel_diff(g.ctrl(), st.P) <= TOL_FP64
    finally:
        g.close()


def test_single_subdomain_equals_global_fit():
    Q = inputs.paper_2d(64)
    g = GpuFit(Q, 3, [20, 17], [1, 1], 2)
    try:
        prob = oracle_problem(Q, 3, [20, 17], [1, 1], 2)
        Pg = O.global_fit(prob, Q)
        assert rel_diff(g.ctrl(), Pg) <= TOL_FP64
        rc, rep = g.iterate(3, 1e-14)
        assert rep.dP_rel <= 1e-14
        assert rel_diff(g.ctrl(), Pg) <= TOL_FP64
    finally:
        g.close()


def test_overlap_ge_p_converges_to_global_fit():
    Q = inputs.asymmetric_sinc_1d(400)
    prob = oracle_problem(Q, 3, [80], [5], 3)
    Pg = O.global_fit(prob, Q)
    g = GpuFit(Q, 3, [80], [5], 3)
    try:
        rc, rep = g.iterate(300, 1e-14)
        assert rc == mfa.MFA_OK
        assert rel_diff(g.ctrl(), Pg) <= 1e-9
        assert rep.jump_max <= 1e-10
    finally:
        g.close()


def test_polynomial_reproduction_on_gpu():
    Q = inputs.tensor_polynomial((45, 38), 3, seed=2)
    g = GpuFit(Q, 3, [14, 12], [3, 3], 1)
    try:
        res = g.residual()
        assert res.maxabs_decoded <= 1e-10 * res.data_range
        rc, rep = g.iterate(1)
        assert rep.dP_rel <= 1e-12
    finally:
        g.close()


def test_scattered_decode_and_derivatives():
    Q = inputs.paper_2d(50)
    lo, hi = [-4.0, -4.0], [4.0, 4.0]
    prob = oracle_problem(Q, 3, [16, 15], [2, 2], 3)
    ref = O.schwarz_solve(prob, Q, max_iters=50, tol_dP=1e-13)
    g = GpuFit(Q, 3, [16, 15], [2, 2], 3, lo=lo, hi=hi)
    try:
        g.iterate(50, 1e-13)
        u = inputs.uniform_points(500, 2, seed=9)
        u[:3] = [[0, 0], [1, 1], [0.5, 1.0]]
        x = np.asarray(lo) + u * (np.asarray(hi) - np.asarray(lo))
        for der in [(0, 0), (1, 0), (0, 2), (1, 1), (3, 2)]:
            out = np.empty(len(u))
            g.model.decode_points(np.ascontiguousarray(x), out, der)
            oref = O.scattered_decode(prob, ref["P"], u, der) / (8.0 ** sum(der))
            scale = max(np.abs(oref).max(), 1e-12)
            assert np.abs(out - oref).max() <= 1e-8 * scale, der
    finally:
        g.close()


@pytest.mark.parametrize("p", [2, 3, 5])
def test_scattered_decode_float_float(p):
    """Scattered decode of a mixed-precision model (float-float control
    points and arithmetic) with derivatives, FP64 and FP32 output: equal to
    the oracle's decode of the model's own control points."""
    Q = inputs.paper_2d(50)
    lo, hi = [-4.0, -4.0], [4.0, 4.0]
    prob = oracle_problem(Q, p, [16, 15], [2, 2], 3)
    g = GpuFit(Q.astype(np.float32), p, [16, 15], [2, 2], 3, lo=lo, hi=hi, precision=mfa.MFA_PREC_MIXED)
    try:
        g.iterate(4)
        P = g.ctrl()
        u = inputs.uniform_points(500, 2, seed=9)
        u[:4] = [[0, 0], [1, 1], [0.5, 1.0], [0.25, 0.0]]
        x = np.asarray(lo) + u * (np.asarray(hi) - np.asarray(lo))
        for der in [(0, 0), (1, 0), (0, 2), (1, 1), (p, 1)]:
            out = np.empty(len(u))
            g.model.decode_points(np.ascontiguousarray(x), out, der)
            oref = O.scattered_decode(prob, P, u, der) / (8.0 ** sum(der))
            scale = max(np.abs(oref).max(), 1e-12)
            assert np.abs(out - oref).max() <= 1e-11 * scale, der
        out32 = np.empty(len(u), dtype=np.float32)
        g.model.decode_points(np.ascontiguousarray(x), out32, (0, 0))
        oref = O.scattered_decode(prob, P, u)
        assert np.abs(out32 - oref).max() <= 2e-7 * max(np.abs(oref).max(), 1e-12)
    finally:
        g.close()


def test_mixed_precision_2d_noise():
    """FP32 data passes and control-point iteration; FP64 Gram/Cholesky."""
    Q = inputs.sinc_2d(256, noise=1e-3, seed=0, dtype=np.float32)
    Qd = Q.astype(np.float64)
    prob = oracle_problem(Qd, 3, [64, 64], [4, 4], 2)
    ref = O.schwarz_solve(prob, Qd, max_iters=30, tol_dP=1e-7)
    g = GpuFit(Q, 3, [64, 64], [4, 4], 2, precision=mfa.MFA_PREC_MIXED)
    try:
        g.iterate(30, 1e-6)
        res = g.residual()
        oref = O.residual_stats(prob, Qd, ref["P"])
        rng = float(Qd.max() - Qd.min())
        assert abs(res.rms_decoded - oref["rms"]) <= 0.01 * oref["rms"]
        D = g.decode_grid(np.float64)
        Dref = O.decode_grid(prob, ref["P"])
        assert np.abs(D - Dref).max() <= 1e-5 * rng
    finally:
        g.close()


# ---------------------------------------------------------------------------
# error paths (host-detected, or reported by the device status word)
# ---------------------------------------------------------------------------

def test_layout_rejections():
    h = mfa.Handle(0)
    try:
        Q = np.zeros(100)
        import torch
        q = torch.zeros(100, dtype=torch.float64, device="cuda")
        bad = [
            dict(p=3, nspans=[20], nsub=[10], delta=1),      # cores of 2 spans < p
            dict(p=3, nspans=[200], nsub=[2], delta=1),      # more CPs than points: Schoenberg-Whitney fails
        ]
        for b in bad:
            lay = mfa.make_layout(1, b["p"], [100], b["nspans"], b["nsub"], [b["delta"]])
            with pytest.raises(mfa.MFAError) as e:
                h.encode(q, lay)
            assert e.value.code == mfa.MFA_ERR_LAYOUT
        lay = mfa.make_layout(1, 3, [100], [20], [2], [1], core_spans=[[5, 14]])  # does not sum to nspans
        with pytest.raises(mfa.MFAError):
            h.encode(q, lay)
        lay = mfa.make_layout(1, 9, [100], [20], [2], [1])  # degree above the maximum
        with pytest.raises(mfa.MFAError) as e:
            h.encode(q, lay)
        assert e.value.code == mfa.MFA_ERR_ARG
        lay = mfa.make_layout(1, 3, [0], [20], [2], [1])  # empty grid
        with pytest.raises(mfa.MFAError) as e:
            h.encode(q, lay)
        assert e.value.code == mfa.MFA_ERR_ARG
        del Q
    finally:
        h.close()


def test_nonfinite_input_reported():
    import torch
    Q = inputs.asymmetric_sinc_1d(200)
    Q[77] = np.nan
    h = mfa.Handle(0)
    try:
        q = torch.from_numpy(Q).cuda()
        lay = mfa.make_layout(1, 3, [200], [40], [2], [1])
        m = h.encode(q, lay)
        with pytest.raises(mfa.MFAError) as e:
            m.iterate(1)
        assert e.value.code == mfa.MFA_ERR_NONFINITE
        m.free()
        # the handle stays usable
        Q[77] = 0.0
        m = h.encode(torch.from_numpy(Q).cuda(), lay)
        rc, rep = m.iterate(2)
        assert np.isfinite(rep.dP_rel)
        m.free()
    finally:
        h.close()


def test_residual_on_staged_host_copy_and_pinned_ctrl():
    """A model encoded from host data keeps its device copy: residual(None)
    equals residual(host data); a device-data model has no copy (MFA_ERR_ARG).
    Control points read into a pinned buffer equal ctrl()."""
    import torch
    Q = inputs.gauss_3d((40, 36, 33), seed=3, dtype=np.float32)
    h = mfa.Handle(0)
    try:
        lay = mfa.make_layout(3, 3, [40, 36, 33], [10, 9, 8], [2, 2, 1], [2, 2, 2], mfa.MFA_PREC_MIXED)
        m = h.encode(Q, lay)
        m.iterate(5, 0.0)
        a, b = m.residual(None), m.residual(Q)
        assert (a.rms_decoded, a.maxabs_decoded, a.data_range) == (b.rms_decoded, b.maxabs_decoded, b.data_range)
        buf = torch.empty(mfa.mfa_num_ctrl(m.m), dtype=torch.float64).pin_memory()
        m.ctrl(out=buf)
        assert np.array_equal(buf.numpy(), m.ctrl().ravel())
        m.free()
        md = h.encode(torch.from_numpy(Q).cuda(), lay)
        with pytest.raises(mfa.MFAError) as ei:
            md.residual(None)
        assert ei.value.code == mfa.MFA_ERR_ARG
        md.free()
    finally:
        h.close()


def test_async_control_point_read_beside_residual():
    """mfa_get_ctrl_async fills a pinned buffer beside later stream work: after
    a residual call and mfa_sync it holds exactly what mfa_get_ctrl returns,
    and a second read into another buffer reuses the staging in order."""
    import torch
    Q = inputs.gauss_3d((40, 36, 33), seed=9, dtype=np.float32)
    h = mfa.Handle(0)
    try:
        lay = mfa.make_layout(3, 3, [40, 36, 33], [10, 9, 8], [2, 2, 1], [2, 2, 2], mfa.MFA_PREC_MIXED)
        m = h.encode(Q, lay)
        m.iterate(5, 0.0)
        n = mfa.mfa_num_ctrl(m.m)
        a = torch.empty(n, dtype=torch.float64).pin_memory()
        b = torch.empty(n, dtype=torch.float64).pin_memory()
        m.ctrl_async(a)
        res = m.residual(None)
        m.iterate(1, 0.0)
        m.ctrl_async(b)
        assert h.sync() == mfa.MFA_OK
        assert res.rms_decoded > 0
        ref = m.ctrl().ravel()
        assert np.array_equal(b.numpy(), ref)
        assert not np.array_equal(a.numpy(), ref)  # the read before the extra step
        with pytest.raises(mfa.MFAError):
            m.ctrl_async(torch.empty(n - 1, dtype=torch.float64))
        m.free()
    finally:
        h.close()


def test_plain_per_subdomain_form_equals_batched_fp64():
    """The per-subdomain comparator form (one launch per subdomain and stage,
    data re-read every iteration) runs the same FP64 arithmetic as the
    batched path: identical control points and iteration count, and it
    matches the oracle within the FP64 bar."""
    Q = inputs.gauss_3d((30, 28, 26), seed=5, dtype=np.float32)
    Qd = Q.astype(np.float64)
    nspans, nsub, delta = [8, 7, 6], [2, 2, 2], 2
    g = GpuFit(Q, 3, nspans, nsub, delta)
    h = mfa.Handle(0)
    try:
        rc, rep = g.iterate(30, 1e-10)
        import torch
        m, rc2, rep2 = h.encode_plain(torch.from_numpy(Q).cuda(), g.layout, 30, 1e-10)
        assert rep2.iters == rep.iters and rc2 == rc
        P = m.ctrl()
        assert np.array_equal(P, g.ctrl())
        prob = oracle_problem(Qd, 3, nspans, nsub, delta)
        ref = O.schwarz_solve(prob, Qd, max_iters=30, tol_dP=1e-10)
        assert ref["iters"] == rep2.iters
        assert rel_diff(P, ref["P"]) <= TOL_FP64
        with pytest.raises(mfa.MFAError):
            h.encode_plain(Q, layout_for_mixed(Q, nspans, nsub, delta), 3, 0.0)
        m.free()
    finally:
        g.close()
        h.close()


def layout_for_mixed(Q, nspans, nsub, delta):
    from mfa_cases import layout_for
    return layout_for(Q, 3, nspans, nsub, delta, mfa.MFA_PREC_MIXED)


@pytest.mark.parametrize("dim,p,delta", [(1, 3, 1), (2, 2, 1), (2, 3, 3), (3, 3, 2)])
def test_owner_update_iterates(dim, p, delta):
    """Owner-takes update (Greville owner per axis): every iterate equals the
    oracle's (FP64 path)."""
    shapes = {1: (90,), 2: (40, 36), 3: (22, 20, 18)}
    spans = {1: [24], 2: [10, 9], 3: [8, 7, 6]}
    nsubs = {1: [3], 2: [2, 3], 3: [2, 2, 2]}
    Q = inputs.random_field(shapes[dim], seed=dim + 10 * p)
    _iterate_parity(Q, p, spans[dim], nsubs[dim], delta, iters=4, update="owner")


def test_owner_update_mixed_3d_fused():
    """Owner-takes update on the fused float-float 3-D path: converged control
    points within 1e-9 of the oracle's owner-takes fixed point."""
    Q = inputs.gauss_3d((48, 44, 40), seed=4, dtype=np.float32)
    Qd = Q.astype(np.float64)
    nspans, nsub, delta = [16, 14, 12], [2, 2, 2], 2
    prob = oracle_problem(Qd, 3, nspans, nsub, delta)
    # stop well above the float-float rounding floor of dP (about 1e-13)
    ref = O.schwarz_solve(prob, Qd, max_iters=60, tol_dP=1e-10, update="owner")
    g = GpuFit(Q, 3, nspans, nsub, delta, precision=mfa.MFA_PREC_MIXED)
    try:
        g.model.set_update_rule(mfa.MFA_UPDATE_OWNER)
        rc, rep = g.iterate(60, 1e-10)
        assert rep.iters == ref["iters"]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
    finally:
        g.close()



def test_overlap_sweep_on_gpu():
    """The delta = 0..2p sweep of Sec. 3.1.1 (asymmetric sinc, N = 5, p = 3)
    through the library: each converged fit equals the oracle's, and from
    delta = p on it is the single-subdomain fit."""
    Q = inputs.asymmetric_sinc_1d(501)
    ref = O.global_fit(O.make_problem(3, [501], [40], [1], 0), Q)
    for delta in range(0, 7):
        prob = oracle_problem(Q, 3, [40], [5], delta)
        o = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-13)
        g = GpuFit(Q, 3, [40], [5], delta)
        try:
            rc, rep = g.iterate(400, 1e-13)
            assert rep.iters == o["iters"]
            P = g.ctrl()
            assert rel_diff(P, o["P"]) <= TOL_FP64
            if delta >= 3:
                assert rel_diff(P, ref) <= 1e-11
        finally:
            g.close()


def test_repeat_encode_reuses_layout_plan():
    """A handle keeps the host products of its latest layout; encoding the same
    layout again (device or host data, with other layouts and data in between)
    gives the same control points bit for bit as a fresh handle, and a
    converged fit still matches the oracle."""
    import torch
    QA = inputs.gauss_3d((40, 36, 33), seed=7, dtype=np.float32)
    QB = inputs.gauss_3d((40, 36, 33), seed=8, dtype=np.float32)
    lay = mfa.make_layout(3, 3, [40, 36, 33], [10, 9, 8], [2, 2, 1], [2, 2, 2], mfa.MFA_PREC_MIXED)
    other = mfa.make_layout(3, 3, [40, 36, 33], [9, 9, 8], [2, 1, 2], [1, 2, 2], mfa.MFA_PREC_MIXED)

    def fit(h, Q, layout, on_device=True):
        q = torch.from_numpy(Q).cuda() if on_device else Q
        m = h.encode(q, layout)
        m.iterate(40, 1e-12)
        P = m.ctrl()
        m.free()
        return P

    fresh, fresh2 = mfa.Handle(0), mfa.Handle(0)
    try:
        ref_A, ref_B = fit(fresh, QA, lay), fit(fresh2, QB, lay)
    finally:
        fresh.close()
        fresh2.close()
    h = mfa.Handle(0)
    try:
        assert np.array_equal(fit(h, QA, lay), ref_A)
        assert np.array_equal(fit(h, QB, lay), ref_B)           # same layout, other data
        fit(h, QA, other)                                        # another layout in between
        assert np.array_equal(fit(h, QA, lay), ref_A)
        assert np.array_equal(fit(h, QA, lay, on_device=False), ref_A)  # host data: staged copy in the pool
        assert np.array_equal(fit(h, QA, lay, on_device=False), ref_A)
        prob = oracle_problem(QA.astype(np.float64), 3, [10, 9, 8], [2, 2, 1], 2)
        ref = O.schwarz_solve(prob, QA.astype(np.float64), max_iters=40, tol_dP=1e-12)
        assert rel_diff(ref_A, ref["P"]) <= TOL_FP64
    finally:
        h.close()


@pytest.mark.parametrize("p,npts,nspans,nsub", [
    (3, (28, 24, 192), (7, 6, 48), (1, 1, 2)),
    (2, (28, 24, 192), (7, 6, 48), (1, 1, 2)),
    (4, (30, 32, 160), (8, 8, 40), (1, 2, 1)),
    (5, (60, 36, 264), (12, 6, 44), (2, 1, 1)),
])
def test_fused_projection_split_along_z(p, npts, nspans, nsub):
    """Windows with enough knot spans along z (26 to 44 here) are projected in
    four units per window of whole plane batches (two CTAs may share a
    z-control point; their partial sums are added by the last unit):
    converged control points within 1e-9 of the oracle's, at even and odd
    numbers of basis lanes.  The stop is dP_rel <= 1e-9, as in the other
    mixed-path tests, above the float-float noise of dP."""
    Q = inputs.gauss_3d(npts, seed=20 + p, dtype=np.float32)  # x, y, z sizes
    Qd = Q.astype(np.float64)
    delta = 2
    prob = oracle_problem(Qd, p, list(nspans), list(nsub), delta)
    ref = O.schwarz_solve(prob, Qd, max_iters=60, tol_dP=1e-9)
    g = GpuFit(Q, p, list(nspans), list(nsub), delta, precision=mfa.MFA_PREC_MIXED)
    gh = GpuFit(Q, p, list(nspans), list(nsub), delta, precision=mfa.MFA_PREC_MIXED, on_device=False)
    try:
        rc, rep = g.iterate(60, 1e-9)
        assert rc == mfa.MFA_OK and rep.iters == ref["iters"]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
        # host data cross in z-slabs beside the projection: the same units in
        # the same order, so the fit is bit-identical to the device-data one
        rch, reph = gh.iterate(60, 1e-9)
        assert (rch, reph.iters) == (rc, rep.iters)
        assert np.array_equal(gh.ctrl(), g.ctrl())
        a, b = g.residual(), gh.model.residual(None)
        assert (a.rms_decoded, a.maxabs_decoded, a.data_range) == (b.rms_decoded, b.maxabs_decoded, b.data_range)
    finally:
        g.close()
        gh.close()


def test_plan_cache_keys_on_core_split_contents():
    """Two layouts equal but for their core split (given as arrays) are
    different plans: encoding them alternately through one handle gives each
    the fit a fresh handle gives it, also when the same array object is
    rewritten in place between the calls."""
    import torch
    Q = inputs.gauss_3d((48, 36, 30), seed=12, dtype=np.float32)
    q = torch.from_numpy(Q).cuda()

    def lay(cores_x):
        return mfa.make_layout(3, 3, [48, 36, 30], [12, 9, 8], [2, 1, 1], [2, 2, 2], mfa.MFA_PREC_MIXED,
                               core_spans=[list(cores_x), None, None])

    def fit(h, layout):
        m = h.encode(q, layout)
        m.iterate(30, 1e-10)
        P = m.ctrl()
        m.free()
        return P

    refs = {}
    for c in ((6, 6), (5, 7)):
        hf = mfa.Handle(0)
        try:
            refs[c] = fit(hf, lay(c))
        finally:
            hf.close()
    assert not np.array_equal(refs[(6, 6)], refs[(5, 7)])
    h = mfa.Handle(0)
    try:
        for c in ((6, 6), (5, 7), (6, 6), (5, 7)):
            assert np.array_equal(fit(h, lay(c)), refs[c])
        one = lay((6, 6))
        assert np.array_equal(fit(h, one), refs[(6, 6)])
        one._keep[0][0], one._keep[0][1] = 5, 7  # the same array, rewritten
        assert np.array_equal(fit(h, one), refs[(5, 7)])
    finally:
        h.close()


def test_two_handles_on_two_threads_match_one():
    """Two host threads, each with a handle on its own stream, encoding host
    data (copy stream, slab pipeline), iterating, reading the control points
    asynchronously and taking the residual at the same time: every fit is
    bit-identical to the same fit on one handle."""
    import threading
    import torch
    Q = inputs.gauss_3d((28, 24, 192), seed=31, dtype=np.float32)
    lay = mfa.make_layout(3, 3, [28, 24, 192], [7, 6, 48], [1, 1, 2], [2, 2, 2], mfa.MFA_PREC_MIXED)
    n = None

    def fit(h, out):
        m = h.encode(Q, lay)
        m.iterate(30, 1e-9)
        m.ctrl_async(out)
        r = m.residual(None)
        assert h.sync() == mfa.MFA_OK
        m.free()
        return r.rms_decoded

    h0 = mfa.Handle(0)
    try:
        n = 1
        for a in range(3):
            n *= [7, 6, 48][a] + 3
        ref = torch.empty(n, dtype=torch.float64).pin_memory()
        ref_rms = fit(h0, ref)
    finally:
        h0.close()
    streams = [torch.cuda.Stream() for _ in range(2)]
    hs = [mfa.Handle(0, stream=s.cuda_stream) for s in streams]
    outs = [[torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)] for _ in hs]
    rms = [[None] * 3 for _ in hs]
    errs = []

    def run(i):
        try:
            for k in range(3):
                rms[i][k] = fit(hs[i], outs[i][k])
        except Exception as e:  # reported below
            errs.append(e)

    try:
        ts = [threading.Thread(target=run, args=(i,)) for i in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errs, errs
        for i in range(2):
            for k in range(3):
                assert np.array_equal(outs[i][k].numpy(), ref.numpy())
                assert rms[i][k] == ref_rms
    finally:
        for h in hs:
            h.close()
