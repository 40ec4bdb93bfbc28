"""The layout of every axis (Sec. 2.2) as the CUDA library's host code
builds it, read through the C ABI on the CPU (mfa_axis_layout touches no
device), against the oracle's index sets: integer work, compared exactly.

What must agree, per subdomain: the core spans, the window (core widened by
the overlap delta, clipped), the data points whose parameter lies in the
closed window interval, and the local control points L; per control point,
the Greville owner of the owner-takes update (Sec. 2.3). The library rejects
a layout when some window's collocation matrix fails the Schoenberg-Whitney
condition; the oracle side decides the same question independently, from the
numerical rank of that matrix built with its own Cox-de Boor basis.
"""
import numpy as np
import pytest

from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import build as B


@pytest.fixture(scope="module")
def mfa():
    from paper_2210_06528_gb300 import mfa as M
    M.load(B.build())
    return M


def oracle_rows(M, nspans, p, cores, delta, clamped=False):
    pcs = O.axis_pieces(M, nspans, p, cores, delta, clamped)
    return np.array([[pc.a, pc.b, pc.w0, pc.w1, pc.k0, pc.k1, pc.L.start, len(pc.L), pc.oU, len(pc.U)]
                     for pc in pcs]), pcs


def column_matching_size(nz):
    """Maximum matching of columns to rows over the nonzero entries of a
    boolean matrix (Kuhn's augmenting paths)."""
    rows, cols = nz.shape
    match_row = [-1] * rows  # row -> column

    def augment(c, seen):
        for r in np.flatnonzero(nz[:, c]):
            if not seen[r]:
                seen[r] = True
                if match_row[r] < 0 or augment(match_row[r], seen):
                    match_row[r] = c
                    return True
        return False

    return sum(1 for c in range(cols) if augment(c, [False] * rows))


def windows_full_rank(M, nspans, p, pcs, t=None):
    """Every window's collocation matrix (its data points x its local control
    points) has full column rank, so its least-squares fit is unique. By the
    Schoenberg-Whitney theorem that holds exactly when every local control
    point can be given its own data point inside its support; decided here
    as a maximum bipartite matching over the nonzero entries of the oracle's
    basis matrix (a numerical rank would misjudge the badly conditioned
    windows of about one point per span)."""
    if t is None:
        t = O.clamped_uniform_knots(nspans, p)
    u = O.grid_params(M)
    for pc in pcs:
        N = O.basis_matrix(t, p, u[pc.k0:pc.k1 + 1])[:, pc.L.start:pc.L.stop]
        if column_matching_size(N != 0.0) < N.shape[1]:
            return False
    return True


def random_cores(rng, nspans, nsub, p):
    """Core spans summing to nspans, each >= p when there are interfaces."""
    lo = p if nsub > 1 else 1
    extra = nspans - lo * nsub
    cuts = np.sort(rng.integers(0, extra + 1, size=nsub - 1))
    parts = np.diff(np.r_[0, cuts, extra])
    return [int(lo + x) for x in parts]


@pytest.mark.parametrize("M,nspans,p,nsub,delta", [(1024, 128, 3, 4, 2), (1024, 256, 3, 4, 2), (512, 192, 3, 8, 2),
                                                   (384, 144, 3, 6, 2), (1024, 128, 3, 4, 0), (501, 40, 3, 5, 6)])
def test_workload_axes_match_oracle(mfa, M, nspans, p, nsub, delta):
    rows, owner = mfa.mfa_axis_layout(M, nspans, p, nsub, delta)
    cores = O.even_cores(nspans, nsub)
    want, pcs = oracle_rows(M, nspans, p, cores, delta)
    assert np.array_equal(rows, want)
    prob = O.make_problem(p, [M], [nspans], [nsub], delta)
    assert np.array_equal(owner, O.greville_owner(prob, 0))


def test_random_layouts_match_oracle(mfa):
    rng = np.random.default_rng(7)
    accepted = rejected = 0
    for _ in range(400):
        p = int(rng.integers(1, 6))
        M = int(rng.integers(2, 300))
        # spans up to about half the points, or (every third draw) up to
        # past the point count, where windows start to lack data
        top = M + 8 if rng.integers(0, 3) == 0 else max(2, M // 2 + 8)
        nspans = int(rng.integers(1, top))
        nsub = int(rng.integers(1, max(2, min(6, nspans // p) + 1)))
        if nsub > 1 and nspans < p * nsub:
            nsub = 1
        delta = int(rng.integers(0, 2 * p + 1))
        cores = random_cores(rng, nspans, nsub, p)
        want, pcs = oracle_rows(M, nspans, p, cores, delta)
        ok = windows_full_rank(M, nspans, p, pcs)
        try:
            rows, owner = mfa.mfa_axis_layout(M, nspans, p, nsub, delta, core_spans=cores)
        except mfa.MFAError as e:
            assert e.code == mfa.MFA_ERR_LAYOUT, (M, nspans, p, cores, delta)
            assert not ok, (M, nspans, p, cores, delta)
            rejected += 1
            continue
        assert ok, (M, nspans, p, cores, delta)
        assert np.array_equal(rows, want), (M, nspans, p, cores, delta)
        prob = O.make_problem(p, [M], [nspans], [nsub], delta, cores=[cores])
        assert np.array_equal(owner, O.greville_owner(prob, 0)), (M, nspans, p, cores, delta)
        accepted += 1
    # the draw covers both outcomes
    assert accepted > 100 and rejected > 20, (accepted, rejected)


def test_random_clamped_layouts_match_oracle(mfa):
    """Clamped interface knots (Sec. 2.2 / Sec. 3.1.1): every interface
    breakpoint repeated p times; the control-point ranges, owners and
    rejections agree with the oracle's layout on that knot vector."""
    rng = np.random.default_rng(17)
    accepted = rejected = 0
    for _ in range(300):
        p = int(rng.integers(1, 6))
        M = int(rng.integers(2, 300))
        top = M + 8 if rng.integers(0, 3) == 0 else max(2, M // 2 + 8)
        nspans = int(rng.integers(1, top))
        nsub = int(rng.integers(1, max(2, min(6, nspans // p) + 1)))
        if nsub > 1 and nspans < p * nsub:
            nsub = 1
        delta = int(rng.integers(0, 2 * p + 1))
        cores = random_cores(rng, nspans, nsub, p)
        want, pcs = oracle_rows(M, nspans, p, cores, delta, clamped=True)
        prob = O.make_problem(p, [M], [nspans], [nsub], delta, cores=[cores], clamped=True)
        ok = windows_full_rank(M, nspans, p, pcs, prob.knots(0))
        try:
            rows, owner = mfa.mfa_axis_layout(M, nspans, p, nsub, delta, core_spans=cores,
                                              knots=mfa.MFA_KNOTS_CLAMPED)
        except mfa.MFAError as e:
            assert e.code == mfa.MFA_ERR_LAYOUT, (M, nspans, p, cores, delta)
            assert not ok, (M, nspans, p, cores, delta)
            rejected += 1
            continue
        assert ok, (M, nspans, p, cores, delta)
        assert np.array_equal(rows, want), (M, nspans, p, cores, delta)
        assert np.array_equal(owner, O.greville_owner(prob, 0)), (M, nspans, p, cores, delta)
        accepted += 1
    assert accepted > 80 and rejected > 10, (accepted, rejected)


def test_rejections(mfa):
    def rc(*args, **kw):
        try:
            mfa.mfa_axis_layout(*args, **kw)
            return mfa.MFA_OK
        except mfa.MFAError as e:
            return e.code
    # a core of fewer than p spans between interfaces
    assert rc(200, 20, 3, 2, 1, core_spans=[2, 18]) == mfa.MFA_ERR_LAYOUT
    # cores that do not add up to the spans
    assert rc(200, 20, 3, 2, 1, core_spans=[9, 10]) == mfa.MFA_ERR_LAYOUT
    # more subdomains than spans
    assert rc(200, 4, 1, 5, 0) == mfa.MFA_ERR_LAYOUT
    # fewer data points than control points (no unique fit)
    assert rc(10, 12, 3, 1, 0) == mfa.MFA_ERR_LAYOUT
    # interpolation: as many control points as points is accepted
    assert rc(15, 12, 3, 1, 0) == mfa.MFA_OK
    # degree and sizes out of range
    assert rc(200, 20, 0, 1, 0) == mfa.MFA_ERR_ARG
    assert rc(200, 20, 8, 1, 0) == mfa.MFA_ERR_ARG
    assert rc(0, 20, 3, 1, 0) == mfa.MFA_ERR_ARG
