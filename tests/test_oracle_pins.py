"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a library routine it does not call
(scipy's B-spline), a brute-force dense computation on explicit Kronecker
matrices, a closed form, or an invariant the paper's method must satisfy.
"""
import numpy as np
import pytest
import scipy.linalg
from scipy.interpolate import BSpline

from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs


# ---------------------------------------------------------------------------
# helpers independent of the oracle: scipy design matrices and Kronecker LSQ
# ---------------------------------------------------------------------------

def scipy_basis(nspans, p, u, deriv=0):
    """Collocation matrix from scipy's own B-spline code (independent of the oracle)."""
    t = np.r_[[0.0] * (p + 1), np.arange(1, nspans) / nspans, [1.0] * (p + 1)]
    n = nspans + p
    if deriv == 0:
        return BSpline.design_matrix(np.asarray(u, float), t, p).toarray()
    return np.stack([BSpline(t, np.eye(n)[i], p).derivative(deriv)(u) for i in range(n)], axis=1)


def kron_axes(mats):
    """Kronecker collocation matrix for arrays of shape (M_{d-1},...,M_0), C order."""
    K = np.ones((1, 1))
    for N in reversed(mats):  # numpy axis 0 = grid axis d-1
        K = np.kron(K, N)
    return K


def uniform_u(M):
    return np.arange(M) / (M - 1) if M > 1 else np.zeros(1)


# ---------------------------------------------------------------------------
# Basis (Sec. 2.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_basis_matches_scipy(p):
    nspans = 9
    rng = np.random.default_rng(p)
    u = np.r_[0.0, 1.0, np.arange(1, nspans) / nspans, rng.uniform(0, 1, 40)]
    t = O.clamped_uniform_knots(nspans, p)
    for r in range(0, p + 1):
        ours = O.basis_matrix(t, p, u, r)
        ref = scipy_basis(nspans, p, u, r)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(ours - ref).max() <= 1e-13 * scale, r


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_partition_of_unity(p):
    nspans = 11
    t = O.clamped_uniform_knots(nspans, p)
    u = np.r_[0.0, 1.0, np.arange(nspans + 1) / nspans, np.random.default_rng(0).uniform(0, 1, 100)]
    N = O.basis_matrix(t, p, u)
    assert np.abs(N.sum(axis=1) - 1.0).max() <= 1e-15 * 4
    assert (N >= -1e-16).all()
    # at most p+1 nonzeros per parameter (local support)
    assert ((np.abs(N) > 0).sum(axis=1) <= p + 1).all()
    for r in range(1, p + 1):
        D = O.basis_matrix(t, p, u, r)
        assert np.abs(D.sum(axis=1)).max() <= 1e-9 * max(1.0, np.abs(D).max())


def test_left_limit_differs_only_in_order_p():
    """At a simple interior knot the one-sided derivatives of orders < p agree
    and the order-p derivative jumps (C^{p-1} basis)."""
    p, nspans = 3, 6
    t = O.clamped_uniform_knots(nspans, p)
    tau = [2 / nspans]
    for r in range(p):
        L = O.basis_matrix(t, p, tau, r, side="left")
        R = O.basis_matrix(t, p, tau, r, side="right")
        assert np.abs(L - R).max() <= 1e-10 * max(1, np.abs(L).max())
    L = O.basis_matrix(t, p, tau, p, side="left")
    R = O.basis_matrix(t, p, tau, p, side="right")
    assert np.abs(L - R).max() > 1.0


# ---------------------------------------------------------------------------
# Layout (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_window_membership_exact():
    """Integer window test agrees with the real-number comparison away from ties,
    and includes both end points on exact ties (closed window)."""
    for M, nspans, delta in [(1024, 128, 2), (101, 20, 3), (64, 16, 1), (17, 16, 2)]:
        pcs = O.axis_pieces(M, nspans, 3, O.even_cores(nspans, 4), delta)
        u = np.arange(M) / (M - 1)
        for pc in pcs:
            lo, hi = pc.w0 / nspans, pc.w1 / nspans
            inside = [k for k in range(M) if lo - 1e-12 <= u[k] <= hi + 1e-12]
            assert pc.k0 == inside[0] and pc.k1 == inside[-1]


def test_layout_two_subdomains_p3_delta1():
    """N=2, p=3, |delta|=1 (the paper's 1-D illustration, Eq. vecp-layout):
    both subdomains own the p control points straddling the interface and each
    holds delta = 1 further control point of its neighbour as frame."""
    pcs = O.axis_pieces(100, 10, 3, [5, 5], 1)
    s0, s1 = pcs
    assert list(s0.U) == list(range(0, 8)) and list(s1.U) == list(range(5, 13))
    assert list(s0.L) == list(range(0, 9)) and list(s1.L) == list(range(4, 13))
    shared = set(s0.U) & set(s1.U)
    assert shared == {5, 6, 7}
    assert set(s0.L) - set(s0.U) == {8} and set(s1.L) - set(s1.U) == {4}


def test_even_cores():
    assert O.even_cores(10, 3) == [4, 3, 3]
    assert O.even_cores(192, 8) == [24] * 8


# ---------------------------------------------------------------------------
# Global LSQ (Eq. minimization-problem) against brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("npts,nspans,p", [((40,), (9,), 3), ((12, 10), (5, 4), 2), ((8, 7, 6), (3, 3, 2), 2),
                                            ((9, 8, 7), (4, 3, 3), 3)])
def test_global_fit_matches_dense_lstsq(npts, nspans, p):
    d = len(npts)
    prob = O.make_problem(p, npts, nspans, [1] * d, 0)
    Q = inputs.random_field(npts, seed=1)
    P = O.global_fit(prob, Q)
    K = kron_axes([scipy_basis(nspans[a], p, uniform_u(npts[a])) for a in range(d)])
    ref = np.linalg.lstsq(K, Q.reshape(-1), rcond=None)[0].reshape(P.shape)
    assert np.abs(P - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_polynomial_reproduction(p):
    """Data from a tensor polynomial of degree <= p lie in the spline space:
    the global fit reproduces them, every local fit is exact, so the first
    averaged iterate is already the fixed point (any delta, any N)."""
    npts, nspans = (41, 23), (12, 9)
    Q = inputs.tensor_polynomial(npts, p, seed=p)
    rng = float(Q.max() - Q.min())
    prob = O.make_problem(p, npts, nspans, [1, 1], 0)
    P = O.global_fit(prob, Q)
    assert O.residual_stats(prob, Q, P)["max"] <= 1e-12 * rng
    for delta in [0, 1, p]:
        prob = O.make_problem(p, npts, nspans, [3, 2], delta)
        st = O.schwarz_initial(prob, Q)
        st1 = O.schwarz_step(prob, Q, st)
        # local normal matrices reach condition ~1e6 at p = 4 with ~3 points
        # per span, so rounding, not the method, sets these bounds
        assert np.abs(st1.P - st.P).max() <= 1e-11 * max(1, np.abs(st.P).max())
        assert O.residual_stats(prob, Q, st1.P)["max"] <= 1e-9 * rng


def test_interpolation_when_n_equals_m():
    """eta = 1: as many control points as data points and N = 1 -> decoded = data."""
    for p in [1, 2, 3, 4]:
        M = 30
        prob = O.make_problem(p, [M], [M - p], [1], 0)
        Q = inputs.symmetric_sinc_1d(M)
        P = O.global_fit(prob, Q)
        assert np.abs(O.decode_grid(prob, P) - Q).max() <= 1e-10


# ---------------------------------------------------------------------------
# Schwarz iteration (Sec. 2.3, Algorithm 1)
# ---------------------------------------------------------------------------

def _converge(prob, Q, tol=1e-14, max_iters=400):
    return O.schwarz_solve(prob, Q, max_iters=max_iters, tol_dP=tol)


@pytest.mark.parametrize("npts,nspans,nsub,p", [((60,), (16,), (3,), 3), ((60,), (16,), (4,), 2),
                                                 ((20, 18), (8, 7), (2, 2), 2), ((11, 10, 9), (6, 5, 4), (2, 2, 1), 2)])
def test_overlap_ge_p_converges_to_global_lstsq(npts, nspans, nsub, p):
    """delta >= p: every owned control point's support lies inside the window,
    so the global LSQ fit (brute-force dense) is the fixed point (Sec. 2.2:
    same error profile as a single subdomain)."""
    d = len(npts)
    Q = inputs.random_field(npts, seed=3)
    prob = O.make_problem(p, npts, nspans, nsub, p)
    res = _converge(prob, Q)
    K = kron_axes([scipy_basis(nspans[a], p, uniform_u(npts[a])) for a in range(d)])
    ref = np.linalg.lstsq(K, Q.reshape(-1), rcond=None)[0].reshape(res["P"].shape)
    assert res["converged"]
    assert np.abs(res["P"] - ref).max() <= 1e-10 * max(1, np.abs(ref).max())
    # and the copies agree: zero jump residual on every shared point
    assert res["history"][-1]["spread"] <= 1e-10 * max(1, np.abs(ref).max())


def _greville_owner_fraction(prob, a):
    """Owner of every control point along axis a by its Greville abscissa,
    computed with exact rationals from the knot vector (independent of the
    oracle's integer sums)."""
    from fractions import Fraction
    p, ns = prob.p, prob.nspans[a]
    t = [Fraction(min(max(i - p, 0), ns), ns) for i in range(ns + 2 * p + 1)]
    pcs = prob.pieces(a)
    own = []
    for g in range(ns + p):
        xi = sum(t[g + 1:g + p + 1]) / p
        i = next(i for i, pc in enumerate(pcs)
                 if Fraction(pc.a, ns) <= xi and (xi < Fraction(pc.b, ns) or (i == len(pcs) - 1 and xi <= 1)))
        own.append(i)
    return own


def _bruteforce_fixed_point(prob, Q, update="average"):
    """Independent construction of the Schwarz fixed point: unknowns are all
    owned copies x_s; equations are the local normal equations of every
    subdomain with its frame equal to the update of the copies (their average,
    or the Greville owner's copy), solved as one dense linear system with
    explicit Kronecker matrices from scipy's basis."""
    d = prob.d
    ncp = prob.ncp()
    gshape = tuple(reversed(ncp))
    G = int(np.prod(ncp))
    subs = prob.subdomains()
    gidx = np.arange(G).reshape(gshape)
    Nfull = [scipy_basis(prob.nspans[a], prob.p, uniform_u(prob.npts[a])) for a in range(d)]
    offs, sizes, ublocks = [], [], []
    n_unk = 0
    for s in subs:
        ug = gidx[tuple(slice(s[a].U.start, s[a].U.stop) for a in reversed(range(d)))].reshape(-1)
        offs.append(n_unk)
        sizes.append(len(ug))
        ublocks.append(ug)
        n_unk += len(ug)
    # update operator W: global P = W x
    W = np.zeros((G, n_unk))
    if update == "average":
        cnt = np.zeros(G)
        for o, ug in zip(offs, ublocks):
            for j, g in enumerate(ug):
                W[g, o + j] = 1.0
                cnt[g] += 1
        W /= cnt[:, None]
    else:
        own = [_greville_owner_fraction(prob, a) for a in range(d)]
        pieces = [prob.pieces(a) for a in range(d)]
        gmulti = np.array(np.unravel_index(np.arange(G), gshape)).T[:, ::-1]  # grid index per axis, axis 0 first
        for o, ug, s in zip(offs, ublocks, subs):
            idx = [pieces[a].index(s[a]) for a in range(d)]
            for j, g in enumerate(ug):
                if all(own[a][gmulti[g][a]] == idx[a] for a in range(d)):
                    W[g, o + j] = 1.0
        assert np.allclose(W.sum(axis=1), 1.0)
    A = np.zeros((n_unk, n_unk))
    b = np.zeros(n_unk)
    for o, ug, s in zip(offs, ublocks, subs):
        pts = [s[a].pts for a in range(d)]
        Lg = gidx[tuple(slice(s[a].L.start, s[a].L.stop) for a in reversed(range(d)))].reshape(-1)
        KL = kron_axes([Nfull[a][pts[a].start:pts[a].stop, s[a].L.start:s[a].L.stop] for a in range(d)])
        qs = Q[tuple(slice(pts[a].start, pts[a].stop) for a in reversed(range(d)))].reshape(-1)
        isU = np.isin(Lg, ug)
        KU, KF = KL[:, isU], KL[:, ~isU]
        Fg = Lg[~isU]
        n = len(ug)
        A[o:o + n, o:o + n] += KU.T @ KU
        A[o:o + n, :] += KU.T @ KF @ W[Fg, :]
        b[o:o + n] += KU.T @ qs
    x = np.linalg.solve(A, b)
    return (W @ x).reshape(gshape)


@pytest.mark.parametrize("npts,nspans,nsub,p,delta", [((60,), (16,), (3,), 3, 1), ((60,), (16,), (3,), 3, 2),
                                                       ((40,), (12,), (3,), 2, 1), ((16, 15), (8, 6), (2, 2), 2, 1),
                                                       ((17, 14), (8, 6), (3, 2), 3, 2)])
def test_overlap_lt_p_fixed_point_bruteforce(npts, nspans, nsub, p, delta):
    """delta < p: the converged iterate equals the fixed point of the averaged
    constrained re-solve, built densely and solved in one shot."""
    Q = inputs.random_field(npts, seed=5)
    prob = O.make_problem(p, npts, nspans, nsub, delta)
    res = _converge(prob, Q)
    ref = _bruteforce_fixed_point(prob, Q)
    assert res["converged"]
    assert np.abs(res["P"] - ref).max() <= 1e-10 * max(1, np.abs(ref).max())


def test_schwarz_step_matches_dense_constrained_lstsq():
    """One constrained re-solve equals a dense LSQ over the owned columns with
    the frame columns moved to the right-hand side (Schur decoupling)."""
    npts, nspans, nsub, p, delta = (17, 14), (8, 6), (3, 2), 3, 2
    d = 2
    Q = inputs.random_field(npts, seed=7)
    prob = O.make_problem(p, npts, nspans, nsub, delta)
    st0 = O.schwarz_initial(prob, Q)
    st1 = O.schwarz_step(prob, Q, st0)
    Nfull = [scipy_basis(nspans[a], p, uniform_u(npts[a])) for a in range(d)]
    for s, copy in zip(prob.subdomains(), st1.copies):
        pts = [s[a].pts for a in range(d)]
        qs = Q[tuple(slice(pts[a].start, pts[a].stop) for a in reversed(range(d)))].reshape(-1)
        KL = kron_axes([Nfull[a][pts[a].start:pts[a].stop, s[a].L.start:s[a].L.stop] for a in range(d)])
        PL = st0.P[tuple(slice(s[a].L.start, s[a].L.stop) for a in reversed(range(d)))]
        mask = np.zeros(PL.shape, bool)
        mask[tuple(slice(s[a].a - s[a].w0, s[a].a - s[a].w0 + len(s[a].U)) for a in reversed(range(d)))] = True
        m = mask.reshape(-1)
        rhs = qs - KL[:, ~m] @ PL.reshape(-1)[~m]
        ref = np.linalg.lstsq(KL[:, m], rhs, rcond=None)[0]
        assert np.abs(copy.reshape(-1) - ref).max() <= 1e-11 * max(1, np.abs(ref).max())


def test_delta_zero_converges_after_one_step():
    """delta = 0: the frame is empty, so every re-solve repeats iteration 0."""
    Q = inputs.paper_2d(41)
    prob = O.make_problem(3, [41, 41], [16, 16], [4, 4], 0)
    res = O.schwarz_solve(prob, Q, max_iters=10, tol_dP=0.0)
    assert res["history"][1]["dP_rel"] == 0.0


def test_single_subdomain_is_global_fit():
    Q = inputs.paper_2d(33)
    for delta in [0, 2]:
        prob = O.make_problem(3, [33, 33], [10, 9], [1, 1], delta)
        res = O.schwarz_solve(prob, Q, max_iters=3, tol_dP=0.0)
        Pg = O.global_fit(prob, Q)
        assert np.abs(res["iterates"] if False else res["P"] - Pg).max() <= 1e-12
        assert res["history"][1]["dP_rel"] <= 1e-15


def test_symmetry_of_double_sinc():
    """sinc(x+1) + sinc(x-1) on [-4,4] is even; a mirror-symmetric layout gives
    mirror-symmetric control points (Sec. 3.1.2)."""
    M = 201
    Q = inputs.symmetric_sinc_1d(M)
    for delta in [0, 2, 3]:
        prob = O.make_problem(3, [M], [40], [5], delta)
        res = O.schwarz_solve(prob, Q, max_iters=200, tol_dP=1e-14)
        P = res["P"]
        assert np.abs(P - P[::-1]).max() <= 1e-12


def test_linearity():
    npts = (25, 22)
    prob = O.make_problem(3, npts, [10, 8], [2, 2], 1)
    Q1, Q2 = inputs.random_field(npts, 1), inputs.random_field(npts, 2)
    f = lambda Q: O.schwarz_solve(prob, Q, max_iters=6, tol_dP=0.0)["P"]
    lhs = f(2.5 * Q1 - 0.75 * Q2)
    rhs = 2.5 * f(Q1) - 0.75 * f(Q2)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_independent_of_subdomain_count_when_overlap_ge_p():
    """With delta >= p the converged control points do not depend on N (Sec. 3.2.4:
    subdomain errors identical across process counts)."""
    M = 257
    Q = inputs.asymmetric_sinc_1d(M)
    ref = None
    for N in [1, 2, 4, 8]:
        prob = O.make_problem(3, [M], [64], [N], 3)
        P = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-14)["P"]
        if ref is None:
            ref = P
        assert np.abs(P - ref).max() <= 1e-10


def test_continuity_at_interfaces():
    """Converged with delta >= p: the local splines of neighbours agree in
    derivative orders 0..p-1 at every interface, the order-p jump stays (C^{p-1})."""
    M, p = 400, 3
    Q = inputs.asymmetric_sinc_1d(M)
    prob = O.make_problem(p, [M], [40], [4], p)
    res = O.schwarz_solve(prob, Q, max_iters=300, tol_dP=1e-15)
    J = O.interface_jumps(prob, res["state"])
    for r in range(p):
        assert J[:, r].max() <= 1e-9
    assert J[:, p].max() > 1e-6
    # the decoupled fit (iteration 0 alone, no constraint) is discontinuous
    st0 = O.schwarz_initial(prob, Q)
    J0 = O.interface_jumps(prob, st0)
    assert J0[:, 0].max() > 1e-9


def test_scattered_decode_matches_grid_decode():
    npts = (13, 11)
    prob = O.make_problem(2, npts, [5, 4], [1, 1], 0)
    P = O.global_fit(prob, inputs.random_field(npts, 4))
    D = O.decode_grid(prob, P)
    u0, u1 = uniform_u(13), uniform_u(11)
    pts = np.array([[u0[i], u1[j]] for j in range(11) for i in range(13)])
    S = O.scattered_decode(prob, P, pts)
    assert np.abs(S - D.reshape(-1)).max() <= 1e-13


# ---------------------------------------------------------------------------
# Owner-takes update (restricted additive Schwarz, Sec. 2.3): every control
# point takes the copy of the subdomain owning its Greville abscissa
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("npts,nspans,nsub,p,delta", [((60,), (16,), (3,), 3, 1), ((40,), (12,), (3,), 2, 1),
                                                       ((16, 15), (8, 6), (2, 2), 2, 1),
                                                       ((17, 14), (8, 6), (3, 2), 3, 2)])
def test_owner_update_fixed_point_bruteforce(npts, nspans, nsub, p, delta):
    Q = inputs.random_field(npts, seed=11)
    prob = O.make_problem(p, npts, nspans, nsub, delta)
    res = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-14, update="owner")
    ref = _bruteforce_fixed_point(prob, Q, update="owner")
    assert res["converged"]
    assert np.abs(res["P"] - ref).max() <= 1e-10 * max(1, np.abs(ref).max())


@pytest.mark.parametrize("npts,nspans,nsub,p,delta", [((70,), (20,), (4,), 3, 3), ((33, 30), (10, 9), (2, 3), 2, 2)])
def test_owner_update_converges_to_global_fit_when_overlap_ge_p(npts, nspans, nsub, p, delta):
    """delta >= p: both update rules share the global LSQ fixed point."""
    Q = inputs.random_field(npts, seed=3)
    prob = O.make_problem(p, npts, nspans, nsub, delta)
    res = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-14, update="owner")
    ref = O.global_fit(prob, Q)
    assert np.abs(res["P"] - ref).max() <= 1e-10 * max(1, np.abs(ref).max())


def test_greville_owner_is_an_owning_subdomain():
    """The Greville abscissa of a control point lies in the core of one of the
    subdomains that own it (its support meets that core), for uneven cores and
    degrees 1..5; and the owner agrees with the exact-rational computation."""
    for p in range(1, 6):
        for cores in ([6, 7, 5], [5, 9], [4, 4, 4, 4]):
            ns = sum(cores)
            if min(cores) < p:
                continue
            prob = O.make_problem(p, [4 * ns + 3], [ns], [len(cores)], 1, cores=[cores])
            own = O.greville_owner(prob, 0)
            assert list(own) == _greville_owner_fraction(prob, 0)
            pcs = prob.pieces(0)
            for g, i in enumerate(own):
                assert g in pcs[i].U


def test_owner_update_single_subdomain_is_the_global_fit():
    Q = inputs.random_field((30, 24), seed=2)
    prob = O.make_problem(3, [30, 24], [9, 7], [1, 1], 0)
    res = O.schwarz_solve(prob, Q, max_iters=3, tol_dP=0.0, update="owner")
    assert np.abs(res["P"] - O.global_fit(prob, Q)).max() <= 1e-12



def test_overlap_sweep_approaches_single_subdomain_fit():
    """Sec. 3.1.1, asymmetric sinc with N = 5 and p = 3: the converged fit
    deviates from the single-subdomain (N = 1) fit less and less as the
    overlap grows from 0 to p - 1 (at least 3x per extra span here), and from
    delta = p up to 2p it is the N = 1 fit itself (reading: with delta >= p
    every owned control point's support lies inside its window)."""
    Q = inputs.asymmetric_sinc_1d(501)
    ref = O.global_fit(O.make_problem(3, [501], [40], [1], 0), Q)
    devs = []
    for delta in range(0, 7):
        prob = O.make_problem(3, [501], [40], [5], delta)
        res = O.schwarz_solve(prob, Q, max_iters=400, tol_dP=1e-14)
        assert res["converged"]
        devs.append(np.abs(res["P"] - ref).max() / np.abs(ref).max())
    for d in range(0, 2):
        assert devs[d + 1] * 3 <= devs[d]
    assert devs[2] > 1e-9
    assert max(devs[3:]) <= 1e-12


@pytest.mark.parametrize("p", [2, 3, 4])
def test_scattered_derivatives_reproduce_polynomial_derivatives(p):
    """Sec. 2.1: a tensor polynomial of per-axis degree <= p lies in the spline
    space, so the global fit reproduces it and every mixed partial derivative
    of the decoded spline equals the polynomial's, computed here in closed
    form from its coefficients. Orders differ per axis and the coefficients
    differ per axis, so a derivative taken along the wrong axis fails."""
    npts, nspans = (23, 19, 17), (5, 4, 3)
    rng = np.random.default_rng(40 + p)
    coef = [rng.standard_normal(p + 1) for _ in range(3)]
    X = np.meshgrid(*[uniform_u(M) for M in reversed(npts)], indexing="ij")  # numpy axis 0 = grid axis 2
    Q = np.ones(X[0].shape)
    for a in range(3):
        Q = Q * np.polynomial.polynomial.polyval(X[2 - a], coef[a])
    prob = O.make_problem(p, npts, nspans, [1, 1, 1], 0)
    P = O.global_fit(prob, Q)
    u = rng.uniform(0.0, 1.0, size=(25, 3))
    u[0] = 0.0
    u[1] = 1.0
    u[2] = [1 / nspans[0], 2 / nspans[1], 1 / nspans[2]]  # on interior breakpoints
    for order in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 2), (2, 0, 1), (1, 1, 1), (p, 0, 0), (0, 2, p)]:
        ours = O.scattered_decode(prob, P, u, deriv=order)
        ref = np.ones(len(u))
        for a in range(3):
            c = np.polynomial.polynomial.polyder(coef[a], order[a]) if order[a] else coef[a]
            ref = ref * np.polynomial.polynomial.polyval(u[:, a], c)
        scale = max(1.0, np.abs(ref).max()) * (p * max(nspans)) ** sum(order)
        assert np.abs(ours - ref).max() <= 1e-12 * scale, order
