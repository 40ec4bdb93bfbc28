"""GPU parity of the decoded-residual stall stop, the interface-jump metric,
clamped interface knots, NURBS weights, FP64 data in the mixed precision,
degrees 6 and 7, and saved models of these layouts -- all through the C ABI
against the FP64 oracle on the same seeded inputs."""
import os
import tempfile

import numpy as np
import pytest

from mfa_cases import TOL_FP64, GpuFit, oracle_problem, rel_diff
from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu

MIXED = mfa.MFA_PREC_MIXED
FP64 = mfa.MFA_PREC_FP64
CLAMPED = mfa.MFA_KNOTS_CLAMPED


def _weights(ncp, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.5, 2.0, n) for n in ncp]


# ---------------------------------------------------------------------------
# decoded-residual stall (Algorithm 1 "check convergence metrics")
# ---------------------------------------------------------------------------

def _oracle_rms_sequence(prob, Q, iters):
    st = O.schwarz_initial(prob, Q)
    rms = [O.residual_stats(prob, Q, st.P)["rms"]]
    for _ in range(iters):
        st = O.schwarz_step(prob, Q, st)
        rms.append(O.residual_stats(prob, Q, st.P)["rms"])
    return rms


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_rms_stall_stop_small(precision):
    """The stop iteration of |RMS_k - RMS_{k-1}| <= tol RMS_k equals the
    oracle's, for a tolerance that separates it from every earlier iteration
    by a wide margin."""
    Q = inputs.paper_2d(97) + 0.01 * inputs.random_field((97, 97), seed=3)
    prob = oracle_problem(Q, 3, [30, 27], [3, 3], 1)
    rms = _oracle_rms_sequence(prob, Q, 12)
    rel = [abs(rms[k] - rms[k - 1]) / rms[k] for k in range(1, len(rms))]
    target = next(k for k in range(3, len(rms)) if rel[k - 1] < min(rel[:k - 1]) / 5)
    tol = np.sqrt(rel[target - 1] * min(rel[:target - 1]))
    ref = O.schwarz_solve(prob, Q, max_iters=50, tol_dP=0.0, tol_rms_stall=tol)
    assert ref["iters"] == target
    g = GpuFit(Q, 3, [30, 27], [3, 3], 1, precision=precision)
    try:
        rc, rep = g.iterate(50, 0.0, tol)
        assert rc == mfa.MFA_OK and rep.iters == target
        assert abs(rep.rms_decoded - rms[target]) <= 1e-6 * rms[target]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
    finally:
        g.close()


@pytest.mark.slow
def test_config2_2d_1024_stops_on_rms_stall():
    """The 2-D workload: 1024^2 of sinc(x)sinc(y) + N(0, 1e-3), FP32 data,
    p = 3, 4x4 subdomains of 64 core spans, overlap 2, mixed precision,
    Schwarz to decoded-residual stall |RMS_k - RMS_{k-1}| <= 1e-6 RMS_k:
    the same stop iteration and RMS as the oracle."""
    Q = inputs.sinc_2d(1024)
    Qd = Q.astype(np.float64)
    prob = oracle_problem(Qd, 3, [256, 256], [4, 4], 2)
    ref = O.schwarz_solve(prob, Qd, max_iters=50, tol_dP=0.0, tol_rms_stall=1e-6)
    assert ref["converged"]
    g = GpuFit(Q, 3, [256, 256], [4, 4], 2, precision=MIXED)
    try:
        rc, rep = g.iterate(50, 0.0, 1e-6)
        assert rc == mfa.MFA_OK
        assert rep.iters == ref["iters"]
        oref = O.residual_stats(prob, Qd, ref["P"])
        assert abs(rep.rms_decoded - oref["rms"]) <= 0.01 * oref["rms"]
        assert abs(rep.rms_decoded - oref["rms"]) <= 1e-7 * oref["rms"]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
    finally:
        g.close()


def test_rms_stall_needs_the_encoded_data():
    """A model loaded from a file has no data to decode against."""
    Q = inputs.paper_2d(41)
    g = GpuFit(Q, 3, [12, 12], [2, 2], 1)
    try:
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "m.mfa")
            g.model.save(path, state=True)
            m2 = g.handle.load(path)
            with pytest.raises(mfa.MFAError) as e:
                m2.iterate(3, 0.0, 1e-6)
            assert e.value.code == mfa.MFA_ERR_ARG
            m2.free()
    finally:
        g.close()


# ---------------------------------------------------------------------------
# interface jumps (Sec. 2.2: C^0 .. C^{p-1})
# ---------------------------------------------------------------------------

def _iterate_tol(Q, p, precision, clamped):
    """Control-point tolerance of an unconverged iterate.  The fused 3-D mixed
    Schwarz step (degrees 2..5, floating knots) solves for its correction in
    FP32 (iterative refinement on a float-float residual), so an iterate
    carries the FP32 rounding of its last correction, about 1e-8 relative,
    which the next step removes; converged, it meets the FP64 bar.  Every
    other path keeps 1e-9 at every iterate."""
    if precision == MIXED and Q.ndim == 3 and not clamped and 2 <= p <= 5:
        return 1e-6
    return TOL_FP64


def _jump_parity(Q, p, nspans, nsub, delta, precision, iters, clamped=False, weights=None):
    knots = CLAMPED if clamped else mfa.MFA_KNOTS_FLOATING
    prob = oracle_problem(Q, p, nspans, nsub, delta, clamped=clamped, weights=weights)
    g = GpuFit(Q, p, nspans, nsub, delta, precision=precision, knots=knots, weights=weights)
    scale = max(1.0, float(np.abs(Q).max()))
    tol = _iterate_tol(Q, p, precision, clamped) * 10
    try:
        st = O.schwarz_initial(prob, Q)
        for k in range(iters + 1):
            if k > 0:
                st = O.schwarz_step(prob, Q, st)
                g.iterate(1)
            J = O.interface_jumps(prob, st, p).max(axis=0)
            got = g.model.jumps(p)
            assert got.shape == (p + 1,)
            assert np.abs(got - J).max() <= (1e-9 if k == 0 else tol) * scale, (k, got, J)
        # converged: the FP64 bar on every path
        ref = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-13)
        g.iterate(300, 1e-13)
        J = O.interface_jumps(prob, ref["state"], p).max(axis=0)
        got = g.model.jumps(p)
        assert np.abs(got - J).max() <= 1e-9 * scale, ("converged", got, J)
        return got
    finally:
        g.close()


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_jumps_2d(precision):
    Q = inputs.paper_2d(97)
    _jump_parity(Q, 3, [30, 27], [3, 3], 1, precision, iters=2)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_jumps_3d(precision):
    Q = inputs.paper_3d(29)
    _jump_parity(Q, 3, [12, 11, 10], [2, 2, 2], 2, precision, iters=2)


def test_jumps_1d_and_converged_continuity():
    """Converged with overlap >= p: every order below p agrees across the
    interfaces, the order-p jump stays (C^{p-1})."""
    Q = inputs.asymmetric_sinc_1d(400)
    _jump_parity(Q, 3, [40], [4], 1, FP64, iters=2)
    g = GpuFit(Q, 3, [40], [4], 3)
    try:
        g.iterate(300, 1e-15)
        J = g.model.jumps(3)
        assert J[:3].max() <= 1e-9 and J[3] > 1e-6
    finally:
        g.close()


def test_jumps_single_subdomain_and_bad_order():
    Q = inputs.paper_2d(41)
    g = GpuFit(Q, 3, [12, 12], [1, 1], 1)
    try:
        assert np.array_equal(g.model.jumps(2), np.zeros(3))
        with pytest.raises(mfa.MFAError):
            g.model.jumps(4)
    finally:
        g.close()


# ---------------------------------------------------------------------------
# clamped interface knots (Sec. 2.2; Sec. 3.1.1, Eq. 1d-asymmetric-sinc)
# ---------------------------------------------------------------------------

def _variant_iterates(Q, p, nspans, nsub, delta, precision, iters, clamped=False, weights=None, derivs=((0,),),
                      tol=None):
    knots = CLAMPED if clamped else mfa.MFA_KNOTS_FLOATING
    prob = oracle_problem(Q, p, nspans, nsub, delta, clamped=clamped, weights=weights)
    g = GpuFit(Q, p, nspans, nsub, delta, precision=precision, knots=knots, weights=weights)
    bar = TOL_FP64 if tol is None else tol
    tol = max(_iterate_tol(Q, p, precision, clamped), bar)
    try:
        st = O.schwarz_initial(prob, Q)
        assert rel_diff(g.ctrl(), st.P) <= bar, "iteration 0"
        for k in range(1, iters + 1):
            st = O.schwarz_step(prob, Q, st)
            rc, rep = g.iterate(1)
            assert rel_diff(g.ctrl(), st.P) <= tol, f"iteration {k}"
            assert abs(rep.jump_max - st.history[-1]["spread"]) <= 10 * tol * max(1, np.abs(st.P).max())
        # converge both sides, then the FP64 bar on every path
        ref = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-13)
        st = ref["state"]
        g.iterate(300, 1e-13)
        assert rel_diff(g.ctrl(), st.P) <= bar, "converged"
        res = g.residual()
        ref = O.residual_stats(prob, Q, st.P)
        scale = max(1.0, float(np.abs(Q).max()))
        assert abs(res.rms_decoded - ref["rms"]) <= 1e-8 * ref["rms"] + 1e-12 * scale
        D = g.decode_grid()
        assert np.abs(D - O.decode_grid(prob, st.P)).max() <= max(1e-10, bar) * scale
        # scattered values and derivatives (parameters = physical coordinates
        # on [0, 1]); a derivative's difference may not exceed what the
        # measured control-point difference propagates to it: that difference
        # times the L1 norm of the point's basis row (derivative rows grow like
        # nspans^r), plus a rounding floor
        d = Q.ndim
        u = np.random.default_rng(5).uniform(0, 1, (64, d))
        Pg = g.ctrl()
        dP = max(rel_diff(Pg, st.P), 1e-15) * np.abs(st.P).max()
        for der in derivs:
            der = list(der) + [0] * (d - len(der))
            out = np.empty(len(u))
            g.model.decode_points(np.ascontiguousarray(u), out, der)
            want = O.scattered_decode(prob, st.P, u, der)
            amp = np.ones(len(u))
            for a in range(d):
                amp *= np.array([np.abs(prob.basis_at(a, [u[k, a]], der[a])).sum() for k in range(len(u))])
            allowed = 10 * dP * amp + 1e-12 * (1 + np.abs(want))
            assert (np.abs(out - want) <= allowed).all(), (der, np.abs(out - want).max(), allowed.min())
        return g.model.jumps(min(p, 2))
    finally:
        g.close()


@pytest.mark.parametrize("delta", [0, 3])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_clamped_asymmetric_sinc_n2(delta, precision):
    """Sec. 3.1.1: N = 2, p = 3, overlap 0 and 3 on Eq. 1d-asymmetric-sinc."""
    Q = inputs.asymmetric_sinc_1d(1000)
    _variant_iterates(Q, 3, [24], [2], delta, precision, iters=4, clamped=True, derivs=((0,), (1,), (2,)))


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_clamped_2d(precision):
    Q = inputs.paper_2d(97)
    _variant_iterates(Q, 3, [30, 27], [3, 2], 1, precision, iters=3, clamped=True, derivs=((0, 0), (1, 0), (1, 1)))


def test_clamped_3d_mixed_uneven():
    Q = inputs.paper_3d(29)
    _variant_iterates(Q, 2, [12, 11, 10], [2, 2, 2], 1, MIXED, iters=2, clamped=True, derivs=((0, 0, 0), (0, 1, 0)))


def test_clamped_is_c0_on_the_gpu():
    """The converged clamped fit: neighbours agree in value at the interface,
    not in slope (GPU jumps of the local splines)."""
    Q = inputs.asymmetric_sinc_1d(1000)
    g = GpuFit(Q, 3, [24], [2], 3, knots=CLAMPED)
    try:
        rc, rep = g.iterate(200, 1e-14)
        assert rc == mfa.MFA_OK
        J = g.model.jumps(1)
        assert J[0] <= 1e-10
        # the local splines share the interface control point's value; the
        # global spline's slope jump is what makes it C^0 only (oracle pin)
    finally:
        g.close()


# ---------------------------------------------------------------------------
# NURBS weights (Eq. nurbs-basis, Sec. 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_nurbs_2d(precision):
    Q = inputs.paper_2d(97)
    W = _weights([30 + 3, 27 + 3], 1)
    _variant_iterates(Q, 3, [30, 27], [3, 2], 2, precision, iters=3, weights=W, derivs=((0, 0), (1, 0), (2, 1)))


def test_nurbs_3d_mixed_fused_shape():
    """Floating knots with weights keep the fused 3-D kernels (they read the
    rational basis tables)."""
    Q = inputs.gauss_3d((48, 44, 40), seed=2, dtype=np.float64)
    W = _weights([16 + 3, 15 + 3, 13 + 3], 2)
    _variant_iterates(Q, 3, [16, 15, 13], [2, 2, 2], 2, MIXED, iters=2, weights=W, derivs=((0, 0, 0), (1, 0, 1)))


def test_nurbs_and_clamped_together():
    Q = inputs.paper_2d(97)
    n = [mfa.ncp_of(3, 30, 3, CLAMPED), mfa.ncp_of(3, 27, 2, CLAMPED)]
    W = _weights(n, 4)
    _variant_iterates(Q, 3, [30, 27], [3, 2], 1, FP64, iters=2, clamped=True, weights=W, derivs=((0, 0), (1, 1)))


def test_nurbs_rejects_bad_weights():
    Q = inputs.paper_2d(41)
    W = _weights([15, 15], 0)
    W[1][3] = 0.0
    with pytest.raises(mfa.MFAError) as e:
        GpuFit(Q, 3, [12, 12], [2, 2], 1, weights=W)
    assert e.value.code == mfa.MFA_ERR_ARG


# ---------------------------------------------------------------------------
# FP64 data in the mixed precision (carried exactly, no FP32 rounding)
# ---------------------------------------------------------------------------

def test_mixed_3d_fp64_data_128():
    """FP64 data at the 512^3 workload's per-subdomain shape (128^3, 2x2x2
    subdomains of 24 spans, p = 3, overlap 2): control points within 1e-9 of
    the oracle and decoded RMS within 1 % -- at the rounding level of FP32 the
    data would have lost more than that."""
    Q = inputs.gauss_3d((128, 128, 128), seed=0, dtype=np.float64)
    prob = oracle_problem(Q, 3, [48] * 3, [2] * 3, 2)
    ref = O.schwarz_solve(prob, Q, max_iters=50, tol_dP=1e-7)
    g = GpuFit(Q, 3, [48] * 3, [2] * 3, 2, precision=MIXED)
    try:
        rc, rep = g.iterate(50, 1e-7)
        assert rep.iters == ref["iters"]
        assert rel_diff(g.ctrl(), ref["P"]) <= TOL_FP64
        res = g.residual()
        oref = O.residual_stats(prob, Q, ref["P"])
        assert abs(res.rms_decoded - oref["rms"]) <= 1e-6 * oref["rms"]
        assert abs(res.maxabs_decoded - oref["max"]) <= 1e-6 * oref["max"]
    finally:
        g.close()


# ---------------------------------------------------------------------------
# degrees 6 and 7 (the paper's Nek5000 study uses p = 6, Sec. 3.2.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [6, 7])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_high_degree_1d_2d(p, precision):
    Q1 = inputs.asymmetric_sinc_1d(601)
    _variant_iterates(Q1, p, [60], [4], 2, precision, iters=3, derivs=((0,), (3,)))
    Q2 = inputs.paper_2d(121)
    _variant_iterates(Q2, p, [30, 28], [2, 2], p, precision, iters=2, derivs=((0, 0), (1, 2)))


def _solve_order_sensitivity(prob, Q):
    """How much the iteration-0 control points move between two correct FP64
    evaluations: the oracle's (Cholesky, axes 0, 1, 2) and LU solves of the
    same normal equations in the order 2, 1, 0.  High degrees make the local
    normal matrices badly conditioned (a window-edge control point's basis
    values are of the order of 1/p! on the window's data), and this measures
    the resulting rounding sensitivity of the problem itself."""
    import scipy.linalg
    Nglob = [prob.basis(a) for a in range(prob.d)]
    copies = []
    for s in prob.subdomains():
        mats = [Nglob[a][s[a].pts.start:s[a].pts.stop, s[a].L.start:s[a].L.stop] for a in range(prob.d)]
        T = O.box(Q, [pc.pts for pc in s])
        for a, N in enumerate(mats):
            T = O.apply_along_axis(T, N.T, a)
        for a in reversed(range(prob.d)):
            A = mats[a].T @ mats[a]
            T = O.apply_along_axis(T, scipy.linalg.solve(A, np.eye(A.shape[0])), a)
        copies.append(O.box(T, [range(pc.oU, pc.oU + len(pc.U)) for pc in s]).copy())
    P2, _ = O.average_copies(prob, prob.subdomains(), copies)
    return rel_diff(P2, O.schwarz_initial(prob, Q).P)


@pytest.mark.parametrize("p", [6, 7])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_high_degree_3d(p, precision):
    """Degrees 6 and 7 in 3-D with overlap p (every owned control point's
    support inside its window).  Tolerance: the FP64 bar, or 20x the problem's
    own FP64 solve-order sensitivity when that is larger (about 1e-9 at p = 7
    here), times 32 for float-float's unit (2^-48 against 2^-53)."""
    Q = inputs.gauss_3d((61, 57, 53), seed=p, dtype=np.float32).astype(np.float64)
    prob = oracle_problem(Q, p, [16, 14, 14], [2, 2, 2], p)
    sigma = _solve_order_sensitivity(prob, Q)
    tol = max(TOL_FP64, 20 * sigma * (32 if precision == MIXED else 1))
    assert tol <= 1e-6, sigma
    _variant_iterates(Q, p, [16, 14, 14], [2, 2, 2], p, precision, iters=2, derivs=((0, 0, 0), (1, 0, 2)), tol=tol)


# ---------------------------------------------------------------------------
# saved models of the variants
# ---------------------------------------------------------------------------

def test_save_load_clamped_nurbs_with_state():
    Q = inputs.paper_2d(97)
    n = [mfa.ncp_of(3, 30, 3, CLAMPED), mfa.ncp_of(3, 27, 2, CLAMPED)]
    W = _weights(n, 6)
    g = GpuFit(Q, 3, [30, 27], [3, 2], 1, precision=MIXED, knots=CLAMPED, weights=W)
    try:
        g.iterate(2)
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "m.mfa")
            g.model.save(path, state=True)
            lay = mfa.saved_layout(path)
            assert lay.knots == CLAMPED
            m2 = g.handle.load(path)
            assert np.array_equal(m2.ctrl(), g.ctrl())
            assert np.array_equal(m2.jumps(3), g.model.jumps(3))
            g.iterate(2)
            m2.iterate(2)
            assert np.array_equal(m2.ctrl(), g.ctrl())
            m2.free()
    finally:
        g.close()
