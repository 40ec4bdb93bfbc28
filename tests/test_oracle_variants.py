"""Pins of the oracle's residual statistics, its decoded-residual stall stop,
its interface-jump metric, the clamped-interface variant and NURBS weights.

Every expected value here comes from something other than the oracle: dense
Kronecker matrices built from scipy's B-spline code, numpy's least squares, an
explicitly iterated dense form of the Schwarz map, finite differences, or a
closed form.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs


# ---------------------------------------------------------------------------
# independent helpers (scipy design matrices, Kronecker products)
# ---------------------------------------------------------------------------

def uniform_u(M):
    return np.arange(M) / (M - 1) if M > 1 else np.zeros(1)


def floating_knots(nspans, p):
    return np.r_[[0.0] * (p + 1), np.arange(1, nspans) / nspans, [1.0] * (p + 1)]


def clamped_interface_knots(nspans, p, cores):
    """Knot vector with the interface breakpoints repeated p times, built from
    the breakpoint list (independent of the oracle's integer construction)."""
    ifaces = np.cumsum(cores)[:-1]
    interior = []
    for i in range(1, nspans):
        interior += [i / nspans] * (p if i in ifaces else 1)
    return np.r_[[0.0] * (p + 1), interior, [1.0] * (p + 1)]


def design(t, p, u, deriv=0):
    """scipy collocation matrix (derivatives through BSpline.derivative)."""
    u = np.asarray(u, float)
    n = len(t) - p - 1
    if deriv == 0:
        return BSpline.design_matrix(u, t, p).toarray()
    return np.stack([BSpline(t, np.eye(n)[i], p).derivative(deriv)(u) for i in range(n)], axis=1)


def kron_axes(mats):
    K = np.ones((1, 1))
    for N in reversed(mats):
        K = np.kron(K, N)
    return K


def kron_vec(vs):
    v = np.ones(1)
    for w in reversed(vs):
        v = np.kron(v, w)
    return v


# ---------------------------------------------------------------------------
# residual statistics (Algorithm 1 "update local error")
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("npts,nspans,p", [((40,), (9,), 3), ((13, 11), (5, 4), 2), ((9, 8, 7), (3, 3, 2), 2)])
def test_residual_stats_on_known_orthogonal_error(npts, nspans, p):
    """Q = R P* + e with e orthogonal to the column space of R: the fit returns
    P*, and the decoded error of P* is e itself, so its RMS is sqrt(mean(e^2))
    and its max is max|e|."""
    d = len(npts)
    K = kron_axes([design(floating_knots(nspans[a], p), p, uniform_u(npts[a])) for a in range(d)])
    rng = np.random.default_rng(11)
    Pstar = rng.normal(size=K.shape[1])
    r = rng.normal(size=K.shape[0])
    e = r - K @ np.linalg.lstsq(K, r, rcond=None)[0]
    Q = (K @ Pstar + e).reshape(tuple(reversed(npts)))
    prob = O.make_problem(p, npts, nspans, [1] * d, 0)
    P = O.global_fit(prob, Q)
    assert np.abs(P.reshape(-1) - Pstar).max() <= 1e-11 * np.abs(Pstar).max()
    st = O.residual_stats(prob, Q, Pstar.reshape(P.shape))
    assert abs(st["rms"] - math.sqrt(np.mean(e * e))) <= 1e-13 * math.sqrt(np.mean(e * e)) + 1e-15
    assert abs(st["max"] - np.abs(e).max()) <= 1e-13 * np.abs(e).max() + 1e-15


# ---------------------------------------------------------------------------
# decoded-residual stall stop (Algorithm 1 "check convergence metrics")
# ---------------------------------------------------------------------------

def _dense_schwarz_iterates(npts, nspans, nsub, p, delta, Q, iters):
    """Algorithm 1 iterated with explicit dense matrices: iteration 0 solves
    every window's LSQ with all local control points free, later iterations
    solve for the owned points with the others fixed at the previous global
    iterate, and the global iterate averages the owned copies."""
    d = len(npts)
    prob = O.make_problem(p, npts, nspans, nsub, delta)  # index sets only
    subs = prob.subdomains()
    ncp = [nspans[a] + p for a in range(d)]
    gshape = tuple(reversed(ncp))
    gidx = np.arange(int(np.prod(ncp))).reshape(gshape)
    Nf = [design(floating_knots(nspans[a], p), p, uniform_u(npts[a])) for a in range(d)]
    Kg = kron_axes(Nf)
    q = Q.reshape(-1)
    Ps, rms = [], []
    P = None
    for k in range(iters + 1):
        acc = np.zeros(gidx.size)
        cnt = np.zeros(gidx.size)
        for s in subs:
            pts = [s[a].pts for a in range(d)]
            KL = kron_axes([Nf[a][pts[a].start:pts[a].stop, s[a].L.start:s[a].L.stop] for a in range(d)])
            qs = Q[tuple(slice(pts[a].start, pts[a].stop) for a in reversed(range(d)))].reshape(-1)
            Lg = gidx[tuple(slice(s[a].L.start, s[a].L.stop) for a in reversed(range(d)))].reshape(-1)
            Ug = gidx[tuple(slice(s[a].U.start, s[a].U.stop) for a in reversed(range(d)))].reshape(-1)
            isU = np.isin(Lg, Ug)
            if k == 0:
                x = np.linalg.lstsq(KL, qs, rcond=None)[0][isU]
            else:
                rhs = qs - KL[:, ~isU] @ P[Lg[~isU]]
                x = np.linalg.lstsq(KL[:, isU], rhs, rcond=None)[0]
            acc[Lg[isU]] += x
            cnt[Lg[isU]] += 1
        P = acc / cnt
        Ps.append(P.copy())
        rms.append(math.sqrt(np.mean((q - Kg @ P) ** 2)))
    return Ps, rms


def test_rms_stall_stop_matches_dense_iteration():
    """The stall rule |RMS_k - RMS_{k-1}| <= tol * RMS_k stops at the first
    iteration k >= 1 where it holds; that iteration is found here from the
    dense iterates, and the oracle must stop there with the same RMS."""
    npts, nspans, nsub, p, delta = (30, 26), (10, 9), (3, 2), 3, 1
    Q = inputs.random_field(npts, seed=9) + inputs.paper_2d(30)[:26, :30]
    Ps, rms = _dense_schwarz_iterates(npts, nspans, nsub, p, delta, Q, 12)
    rel = [abs(rms[k] - rms[k - 1]) / rms[k] for k in range(1, len(rms))]
    # the first iteration k >= 3 whose relative change is 3x below every
    # earlier one, and a tolerance halfway (geometrically) between them
    target = next(k for k in range(3, len(rms)) if rel[k - 1] < min(rel[:k - 1]) / 3)
    tol = math.sqrt(rel[target - 1] * min(rel[:target - 1]))
    stop = next(k for k in range(1, len(rms)) if rel[k - 1] <= tol)
    assert stop == target
    prob = O.make_problem(p, npts, nspans, nsub, delta)
    res = O.schwarz_solve(prob, Q, max_iters=50, tol_dP=0.0, tol_rms_stall=tol)
    assert res["converged"] and res["iters"] == stop
    assert abs(res["history"][-1]["rms"] - rms[stop]) <= 1e-12 * rms[stop]
    assert np.abs(res["P"].reshape(-1) - Ps[stop]).max() <= 1e-11 * np.abs(Ps[stop]).max()


# ---------------------------------------------------------------------------
# interface jumps in 2-D and 3-D (Sec. 2.2, C^0 .. C^{p-1})
# ---------------------------------------------------------------------------

def _local_value(prob, s, X, a, tau, r, knots):
    """A subdomain's local spline (its L box X, zero elsewhere) and its r-th
    derivative along axis a at u_a = tau, sampled along the other axes at the
    data points of its core, through scipy (a single spline is C^{p-1}, so for
    r < p its one-sided limits equal its value)."""
    d = prob.d
    mats = []
    for b in range(d):
        Lr = s[b].L
        if b == a:
            D = design(knots[b], prob.p, [tau], r) / prob.nspans[a] ** r
        else:
            M = prob.npts[b]
            ks = [k for k in range(M) if s[b].a * (M - 1) <= k * prob.nspans[b] <= s[b].b * (M - 1)]
            D = design(knots[b], prob.p, uniform_u(M)[ks])
        mats.append(D[:, Lr.start:Lr.stop])
    return kron_axes(mats) @ X.reshape(-1)


@pytest.mark.parametrize("npts,nspans,nsub,p", [((31, 29), (9, 8), (2, 2), 3), ((14, 13, 12), (6, 6, 5), (2, 2, 1), 2)])
def test_interface_jumps_multi_d(npts, nspans, nsub, p):
    d = len(npts)
    Q = inputs.random_field(npts, seed=2)
    knots = [floating_knots(nspans[a], p) for a in range(d)]
    # iteration 0 (no constraint): jumps of orders < p equal the scipy values
    prob = O.make_problem(p, npts, nspans, nsub, 1)
    st0 = O.schwarz_initial(prob, Q)
    J0 = O.interface_jumps(prob, st0, p - 1)
    subs = prob.subdomains()
    pieces = [prob.pieces(a) for a in range(d)]
    row = 0
    for a in range(d):
        for i, s in enumerate(subs):
            if pieces[a].index(s[a]) + 1 >= len(pieces[a]):
                continue
            j = next(j for j, t in enumerate(subs)
                     if all((pieces[b].index(t[b]) == pieces[b].index(s[b]) + (1 if b == a else 0)) for b in range(d)))
            tau = s[a].b / nspans[a]
            for r in range(p):
                vl = _local_value(prob, s, st0.frames[i], a, tau, r, knots)
                vr = _local_value(prob, subs[j], st0.frames[j], a, tau, r, knots)
                ref = np.abs(vl - vr).max()
                assert abs(J0[row, r] - ref) <= 1e-10 * max(1.0, ref), (a, i, r)
            row += 1
    assert row == J0.shape[0] and J0[:, 0].max() > 1e-6
    # converged with delta >= p: C^{p-1} across every interface, order p jumps
    prob = O.make_problem(p, npts, nspans, nsub, p)
    res = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-15)
    J = O.interface_jumps(prob, res["state"])
    assert J[:, :p].max() <= 1e-9
    assert J[:, p].max() > 1e-4


# ---------------------------------------------------------------------------
# clamped interface knots (Sec. 2.2, Sec. 3.1.1)
# ---------------------------------------------------------------------------

def test_clamped_knots_and_layout():
    p, nspans, cores = 3, 12, [4, 5, 3]
    prob = O.make_problem(p, [61], [nspans], [3], 1, cores=[cores], clamped=True)
    t = prob.knots(0)
    assert np.array_equal(t, clamped_interface_knots(nspans, p, cores))
    assert prob.ncp() == [nspans + p + (p - 1) * 2]
    pcs = prob.pieces(0)
    # every core owns its own clamped basis: c + p control points; neighbours
    # share exactly the one control point at their interface
    for pc, c in zip(pcs, cores):
        assert len(pc.U) == c + p
    for l, r in zip(pcs[:-1], pcs[1:]):
        assert set(l.U) & set(r.U) == {l.U.stop - 1} and r.U.start == l.U.stop - 1
    # the frame is delta = 1 span of the neighbour: its p further control points
    assert pcs[0].L.stop - pcs[0].U.stop == p and pcs[1].U.start - pcs[1].L.start == p


def _local_fit(u, q, lo, hi, c, p):
    """Fit data at parameters u in [lo, hi] with the core's own clamped
    uniform knots (c spans), by dense least squares through scipy."""
    v = (u - lo) / (hi - lo)
    N = design(floating_knots(c, p), p, np.clip(v, 0.0, 1.0))
    return np.linalg.lstsq(N, q, rcond=None)[0]


def test_clamped_delta0_is_averaged_independent_fits():
    """delta = 0: every core is fitted on its own with clamped local knots
    (Sec. 2.2: the interface control point interpolates there), and the shared
    interface control point is the average of the two fits."""
    M, p, nspans, cores = 201, 3, 20, [7, 6, 7]
    Q = inputs.asymmetric_sinc_1d(M)
    prob = O.make_problem(p, [M], [nspans], [3], 0, cores=[cores], clamped=True)
    res = O.schwarz_solve(prob, Q, max_iters=3, tol_dP=0.0)
    u = uniform_u(M)
    acc = np.zeros(prob.ncp()[0])
    cnt = np.zeros_like(acc)
    for pc in prob.pieces(0):
        lo, hi = pc.a / nspans, pc.b / nspans
        ks = [k for k in range(M) if lo - 1e-15 <= u[k] <= hi + 1e-15]
        x = _local_fit(u[ks], Q[ks], lo, hi, pc.b - pc.a, p)
        acc[pc.U.start:pc.U.stop] += x
        cnt[pc.U.start:pc.U.stop] += 1
    ref = acc / cnt
    assert np.abs(res["P"] - ref).max() <= 1e-11 * np.abs(ref).max()
    assert res["history"][1]["dP_rel"] == 0.0


@pytest.mark.parametrize("npts,nspans,nsub,p,delta", [((120,), (24,), (3,), 3, 1), ((120,), (24,), (4,), 2, 2),
                                                       ((41, 37), (12, 10), (2, 2), 3, 1),
                                                       ((13, 12, 11), (6, 6, 4), (2, 2, 1), 2, 1)])
def test_clamped_overlap_converges_to_global_fit_on_repeated_knots(npts, nspans, nsub, p, delta):
    """delta >= 1: the supports of the owned control points lie inside the
    windows (the interface control point's support is one span on each side),
    so the fixed point is the global LSQ fit on the knot vector with the
    interfaces repeated p times."""
    d = len(npts)
    Q = inputs.random_field(npts, seed=4)
    prob = O.make_problem(p, npts, nspans, nsub, delta, clamped=True)
    res = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-15)
    K = kron_axes([design(clamped_interface_knots(nspans[a], p, prob.cores[a]), p, uniform_u(npts[a]))
                   for a in range(d)])
    ref = np.linalg.lstsq(K, Q.reshape(-1), rcond=None)[0]
    assert res["converged"]
    assert np.abs(res["P"].reshape(-1) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_clamped_is_c0_only_and_depends_on_n():
    """Sec. 2.2 / 3.1.1: clamped interfaces give a C^0 fit whose first
    derivative jumps at the interfaces, and the fit changes with N; floating
    knots with delta >= p give C^{p-1} and the same fit for every N."""
    M, p = 400, 3
    Q = inputs.asymmetric_sinc_1d(M)
    fits = {}
    for N in (2, 4):
        prob = O.make_problem(p, [M], [40], [N], p, clamped=True)
        res = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-15)
        G = O.global_jumps(prob, res["P"], 2)
        assert G[:, 0].max() <= 1e-12
        assert G[:, 1].min() > 1e-6
        # the local splines of neighbours agree at convergence (shared value)
        assert O.interface_jumps(prob, res["state"], 0).max() <= 1e-10
        fits[N] = O.decode_grid(prob, res["P"])
    assert np.abs(fits[2] - fits[4]).max() > 1e-6
    for N in (2, 4):
        prob = O.make_problem(p, [M], [40], [N], p)
        res = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-15)
        G = O.global_jumps(prob, res["P"], p)
        assert G[:, :p].max() <= 1e-9 and G[:, p].max() > 1e-9
        fits[("f", N)] = O.decode_grid(prob, res["P"])
    assert np.abs(fits[("f", 2)] - fits[("f", 4)]).max() <= 1e-10


def test_clamped_error_below_floating_on_asymmetric_sinc():
    """Sec. 3.1.1 (Eq. 1d-asymmetric-sinc, N = 2, p = 3): the clamped
    subdivision's decoded error is lower than the floating-knot fits' (it has
    p - 1 more control points at the interface), with delta in {0, 3}."""
    M, p, nspans = 1000, 3, 24
    Q = inputs.asymmetric_sinc_1d(M)
    rms = {}
    for clamped in (True, False):
        for delta in (0, 3):
            prob = O.make_problem(p, [M], [nspans], [2], delta, clamped=clamped)
            res = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-14)
            rms[(clamped, delta)] = O.residual_stats(prob, Q, res["P"])["rms"]
    for delta in (0, 3):
        assert rms[(True, delta)] < rms[(False, 0)] and rms[(True, delta)] < rms[(False, 3)], rms


# ---------------------------------------------------------------------------
# NURBS weights (Eq. nurbs-basis, Sec. 4)
# ---------------------------------------------------------------------------

def _weights(ncp, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.5, 2.0, n) for n in ncp]


def test_rational_basis_partition_and_unit_weights():
    p, nspans = 3, 7
    t = floating_knots(nspans, p)
    u = np.r_[0.0, 1.0, np.random.default_rng(0).uniform(0, 1, 50)]
    W = np.random.default_rng(1).uniform(0.3, 3.0, nspans + p)
    R = O.rational_basis(t, p, W, u)
    assert np.abs(R.sum(axis=1) - 1).max() <= 1e-14
    for r in (1, 2, 3):
        assert np.abs(O.rational_basis(t, p, W, u, r).sum(axis=1)).max() <= 1e-9 * nspans ** r
    assert np.abs(O.rational_basis(t, p, np.ones(nspans + p), u, 2) - design(t, p, u, 2)).max() <= 1e-10


def test_rational_derivatives_against_finite_differences():
    """Richardson-extrapolated central differences of R inside the spans."""
    p, nspans = 3, 6
    t = floating_knots(nspans, p)
    W = np.random.default_rng(2).uniform(0.5, 2.0, nspans + p)
    u = (np.arange(nspans) + np.array([0.3, 0.55, 0.7, 0.45, 0.62, 0.38])) / nspans
    R = lambda x: O.rational_basis(t, p, W, x)
    for r in (1, 2):
        def fd(h):
            if r == 1:
                return (R(u + h) - R(u - h)) / (2 * h)
            return (R(u + h) - 2 * R(u) + R(u - h)) / (h * h)
        h = 1e-3 / nspans
        est = (4 * fd(h / 2) - fd(h)) / 3
        ref = O.rational_basis(t, p, W, u, r)
        assert np.abs(est - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max()), r


@pytest.mark.parametrize("npts,nspans,p", [((35,), (8,), 3), ((14, 12), (5, 4), 2), ((9, 8, 7), (3, 3, 2), 2)])
def test_nurbs_global_fit_matches_dense_rational_lstsq(npts, nspans, p):
    """The weighted fit minimises ||Q - R P|| with R[k, g] = N_g(u_k) W_g /
    sum_h N_h(u_k) W_h on the full tensor basis (W_g the product of the axis
    weights), built here without using separability."""
    d = len(npts)
    Q = inputs.random_field(npts, seed=6)
    ncp = [nspans[a] + p for a in range(d)]
    W = _weights(ncp, 3)
    prob = O.make_problem(p, npts, nspans, [1] * d, 0, weights=W)
    P = O.global_fit(prob, Q)
    Nk = kron_axes([design(floating_knots(nspans[a], p), p, uniform_u(npts[a])) for a in range(d)])
    A = Nk * kron_vec(W)[None, :]
    Rk = A / A.sum(axis=1, keepdims=True)
    ref = np.linalg.lstsq(Rk, Q.reshape(-1), rcond=None)[0]
    assert np.abs(P.reshape(-1) - ref).max() <= 1e-11 * max(1, np.abs(ref).max())
    # scattered decode equals the dense rational evaluation
    rng = np.random.default_rng(7)
    uq = rng.uniform(0, 1, (9, d))
    val = O.scattered_decode(prob, P, uq)
    for k in range(len(uq)):
        row = kron_axes([design(floating_knots(nspans[a], p), p, [uq[k, a]]) for a in range(d)])[0] * kron_vec(W)
        assert abs(val[k] - row @ ref / row.sum()) <= 1e-11 * max(1, np.abs(ref).max())


def test_nurbs_schwarz_converges_to_weighted_global_fit():
    npts, nspans, nsub, p = (30, 27), (10, 9), (2, 3), 2
    Q = inputs.random_field(npts, seed=8)
    W = _weights([nspans[a] + p for a in range(2)], 5)
    prob = O.make_problem(p, npts, nspans, nsub, p, weights=W)
    res = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-15)
    ref = O.global_fit(O.make_problem(p, npts, nspans, [1, 1], 0, weights=W), Q)
    assert res["converged"]
    assert np.abs(res["P"] - ref).max() <= 1e-10 * np.abs(ref).max()
    J = O.interface_jumps(prob, res["state"])
    assert J[:, :p].max() <= 1e-9
