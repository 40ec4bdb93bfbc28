"""Plain FP64 CPU oracle for the domain-decomposed MFA encoder.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm use it.  It shares no code with the CUDA library.

Paper: Mahadevan, Lenz, Grindeanu, Peterka, "Parallel Domain Decomposition
Techniques Applied to Multivariate Functional Approximation of Discrete Data"
(arXiv 2210.06528).

What it computes, in the paper's order (Algorithm 1):
  * Sec. 2.1, Eq. (nurbs-basis) with W = 1: B-spline basis N_{i,p} by the
    Cox-de Boor recurrence, and its exact derivatives by the same recurrence.
  * Sec. 2.1, Eq. (minimization-problem): the unconstrained local LSQ fit,
    solved through the normal equations with a Cholesky factorisation
    (Sec. 2.3.1).  On a tensor grid the normal matrix is the Kronecker product
    of per-axis Gram matrices, so the solve is applied one axis at a time.
  * Sec. 2.2 (floating interior knots, Delta / delta layers, Eq. vecp-layout)
    and Sec. 2.3 (Eq. nonlinear-residuals, RAS with w_i = 1/n_s): the outer
    additive-Schwarz loop.  Iteration 0 is the decoupled unconstrained solve
    of every subdomain; iteration k >= 1 re-solves every subdomain with its
    frame control points (those it sees in its overlap but does not own) held
    at the lagged global iterate, which is the Schur-complement decoupling of
    Eq. (global-system) with the constraint imposed exactly; the new global
    iterate averages every owned copy with weight 1/n_s.
  * Algorithm 1, "update local error": decode R P and the residual Q - R P.
  * Algorithm 1, "check convergence metrics" and Sec. 2.2 (C^0 .. C^{p-1}):
    one-sided derivative jumps between neighbouring local splines at every
    subdomain interface.
  * Sec. 2.2 and Sec. 3.1.1 (clamped versus floating interface knots): the
    clamped-interface variant repeats every interface breakpoint p times, so
    neighbours share exactly one control point there (C^0 only).
  * Sec. 2.1, Eq. (nurbs-basis) with W != 1 and Sec. 4: rational basis with
    per-axis control-point weights.

Readings where the paper is silent:
  * data parameters u_k = k / (M - 1) on every axis; M = 1 gives u = 0;
  * global knots clamped and uniform: nspans spans, n = nspans + p control
    points; subdomain interfaces sit on breakpoints, so interior knots float;
  * clamped-interface variant: the same breakpoints, each interface breakpoint
    repeated p times (n = nspans + p + (p - 1)(N_a - 1) per axis); inside a
    core this is the core's own clamped uniform knot vector, and the single
    control point at the interface is shared by both neighbours;
  * NURBS weights are separable, W_g = W_0[g_0] W_1[g_1] W_2[g_2], so the
    rational basis is the tensor product of per-axis rational bases and the
    fit stays separable; the weights are fixed inputs, so averaging the
    weighted control points P W equals averaging P;
  * subdomain cores are contiguous span ranges [a, b); a core owns the control
    points whose support meets it, U = [a, b + p);
  * the overlap delta extends the core by delta spans per interior side: the
    window is [a - delta, b + delta) clipped to [0, nspans); the data of a
    subdomain are the points whose parameter lies in the CLOSED window
    interval, decided with exact integer arithmetic;
  * L = all control points touching the window = [w0, w1 + p); the frame is
    F = L minus U (tensor product: any axis index outside U);
  * the converged state is the fixed point of the averaged re-solve map.

Array convention: a d-dimensional grid array has numpy shape
(M_{d-1}, ..., M_1, M_0), C order, so grid axis 0 is the fastest-varying
index in memory.  ``_np_axis(a, d)`` converts grid axis a to numpy axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------
# Sec. 2.1: knots, parameters and the Cox-de Boor basis
# ---------------------------------------------------------------------------


def clamped_uniform_knots(nspans: int, p: int) -> np.ndarray:
    """Clamped uniform knot vector with ``nspans`` spans: p+1 zeros, the
    interior breakpoints i/nspans, p+1 ones (Sec. 2.1; global ends clamped,
    Sec. 2.2; interior knots single, i.e. floating at interfaces)."""
    interior = [i / nspans for i in range(1, nspans)]
    return np.array([0.0] * (p + 1) + interior + [1.0] * (p + 1), dtype=np.float64)


def knot_ints(nspans: int, p: int, cores: Optional[Sequence[int]] = None) -> List[int]:
    """Knot positions in units of one span (t_i = k_i / nspans).  Without
    ``cores`` the clamped uniform vector; with ``cores`` the clamped-interface
    variant (Sec. 2.2): every interface breakpoint between two cores is
    repeated p times (at least once), which makes the spline C^0 there and
    makes its one straddling control point interpolate the interface value."""
    bounds = set()
    if cores is not None:
        acc = 0
        for c in list(cores)[:-1]:
            acc += c
            bounds.add(acc)
    k = [0] * (p + 1)
    for i in range(1, nspans):
        k += [i] * (max(p, 1) if i in bounds else 1)
    return k + [nspans] * (p + 1)


def grid_params(M: int) -> np.ndarray:
    """Uniform data parameters u_k = k/(M-1) (reading: the paper does not fix
    the parameterisation).  A single point sits at u = 0."""
    if M == 1:
        return np.zeros(1)
    return np.arange(M, dtype=np.float64) / (M - 1)


def _degree0(t: np.ndarray, u: np.ndarray, side: str) -> np.ndarray:
    """N_{i,0}(u): indicator of [t_i, t_{i+1}) ('right') or (t_i, t_{i+1}]
    ('left', the left-sided limit).  With side 'right' the global end u = t[-1]
    is assigned to the last non-empty interval, with side 'left' the global
    start u = t[0] to the first one, so the basis is defined on the closed
    parameter interval."""
    m = len(t) - 1
    N = np.zeros((len(u), m))
    for i in range(m):
        if side == "right":
            N[:, i] = (t[i] <= u) & (u < t[i + 1])
        else:
            N[:, i] = (t[i] < u) & (u <= t[i + 1])
    nonempty = [i for i in range(m) if t[i] < t[i + 1]]
    if side == "right":
        N[u == t[-1], nonempty[-1]] = 1.0
    else:
        N[u == t[0], nonempty[0]] = 1.0
    return N


def basis_matrix(t: np.ndarray, p: int, u, deriv: int = 0, side: str = "right") -> np.ndarray:
    """Dense collocation matrix D[k, i] = d^deriv/du^deriv N_{i,p}(u_k).

    Cox-de Boor recurrence (Sec. 2.1, Eq. nurbs-basis with W = 1):
        N_{i,q}(u) = (u - t_i)/(t_{i+q} - t_i) N_{i,q-1}(u)
                   + (t_{i+q+1} - u)/(t_{i+q+1} - t_{i+1}) N_{i+1,q-1}(u),
    with a term dropped when its denominator is zero.  Derivatives use the
    same recurrence on the derivative (Sec. 2.1 notes exact derivatives follow
    from it):
        N^{(r)}_{i,q} = q/(t_{i+q} - t_i) N^{(r-1)}_{i,q-1}
                      - q/(t_{i+q+1} - t_{i+1}) N^{(r-1)}_{i+1,q-1}.
    The matrix has len(t) - p - 1 columns.
    """
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    t = np.asarray(t, dtype=np.float64)
    if deriv > p:
        return np.zeros((len(u), len(t) - p - 1))
    if deriv == 0:
        N = _degree0(t, u, side)
        for q in range(1, p + 1):
            cols = N.shape[1] - 1
            Nq = np.zeros((len(u), cols))
            for i in range(cols):
                d1 = t[i + q] - t[i]
                d2 = t[i + q + 1] - t[i + 1]
                if d1 > 0:
                    Nq[:, i] += (u - t[i]) / d1 * N[:, i]
                if d2 > 0:
                    Nq[:, i] += (t[i + q + 1] - u) / d2 * N[:, i + 1]
            N = Nq
        return N
    lower = basis_matrix(t, p - 1, u, deriv - 1, side)  # columns: len(t) - p
    cols = lower.shape[1] - 1
    D = np.zeros((len(u), cols))
    for i in range(cols):
        d1 = t[i + p] - t[i]
        d2 = t[i + p + 1] - t[i + 1]
        if d1 > 0:
            D[:, i] += p / d1 * lower[:, i]
        if d2 > 0:
            D[:, i] -= p / d2 * lower[:, i + 1]
    return D


def rational_basis(t: np.ndarray, p: int, W: np.ndarray, u, deriv: int = 0, side: str = "right") -> np.ndarray:
    """Rational basis R_i = N_i W_i / sum_j N_j W_j (Sec. 2.1, Eq. nurbs-basis)
    and its derivatives.  With A = sum_i N_i W_i P_i and w = sum_j N_j W_j the
    curve is A / w; differentiating w R = N W r times (Leibniz) gives
        R^(r) = (N^(r) W - sum_{j=1..r} binom(r, j) w^(j) R^(r-j)) / w."""
    W = np.asarray(W, np.float64)
    Nd = [basis_matrix(t, p, u, r, side) for r in range(deriv + 1)]
    w = [N @ W for N in Nd]
    R = []
    for r in range(deriv + 1):
        v = Nd[r] * W[None, :]
        for j in range(1, r + 1):
            v = v - math.comb(r, j) * w[j][:, None] * R[r - j]
        R.append(v / w[0][:, None])
    return R[deriv]


# ---------------------------------------------------------------------------
# Sec. 2.2: subdomain layout along one axis
# ---------------------------------------------------------------------------


@dataclass
class AxisPiece:
    """One subdomain's index sets along one grid axis (Sec. 2.2, Eq. vecp-layout).

    core  [a, b)          : owned knot spans (Omega_i)
    window[w0, w1)        : core plus delta spans per interior side (delta_i)
    pts   [k0, k1]        : data points in the closed window interval
    U     [a, b + p)      : owned control points, P(Omega) and P(Delta)
    L     [w0, w1 + p)    : every control point touching the window
    The control-point ranges are shifted by ``cshift`` (the first control
    point of span j is j + cshift(j)) in the clamped-interface variant, where
    each interface before span j adds p - 1 control points.
    """

    a: int
    b: int
    w0: int
    w1: int
    k0: int
    k1: int
    p: int
    u0: int = -1  # first owned control point (-1: floating knots, a)
    u1: int = -1  # one past the last owned control point
    l0: int = -1
    l1: int = -1

    @property
    def U(self) -> range:
        if self.u0 < 0:
            return range(self.a, self.b + self.p)
        return range(self.u0, self.u1)

    @property
    def L(self) -> range:
        if self.l0 < 0:
            return range(self.w0, self.w1 + self.p)
        return range(self.l0, self.l1)

    @property
    def oU(self) -> int:
        """Offset of U inside L."""
        return self.U.start - self.L.start

    @property
    def pts(self) -> range:
        return range(self.k0, self.k1 + 1)


def even_cores(nspans: int, nsub: int) -> List[int]:
    """Split nspans into nsub contiguous cores; the +1 spans of an uneven split
    go to the first subdomains (reading)."""
    base, extra = divmod(nspans, nsub)
    return [base + (1 if s < extra else 0) for s in range(nsub)]


def axis_pieces(M: int, nspans: int, p: int, core_spans: Sequence[int], delta: int,
                clamped: bool = False) -> List[AxisPiece]:
    """Index sets of every subdomain along one axis.

    Window membership of data point k (parameter k/(M-1)) in the closed
    interval [w0/nspans, w1/nspans] is decided exactly:
        w0 * (M-1) <= k * nspans <= w1 * (M-1).
    With ``clamped`` (interface knots repeated p times) the first control
    point of span j is j + (p - 1) * (number of interfaces at or before j).
    """
    assert sum(core_spans) == nspans
    starts = list(np.cumsum([0] + list(core_spans)))
    ifaces = starts[1:-1]

    def first_cp(j):
        return j + (max(p, 1) - 1) * sum(1 for b in ifaces if b <= j) if clamped else j

    pieces = []
    a = 0
    for c in core_spans:
        b = a + c
        w0 = max(a - delta, 0)
        w1 = min(b + delta, nspans)
        if M == 1:
            k0 = k1 = 0
        else:
            ks = [k for k in range(M) if w0 * (M - 1) <= k * nspans <= w1 * (M - 1)]
            k0, k1 = ks[0], ks[-1]
        if clamped:
            pieces.append(AxisPiece(a, b, w0, w1, k0, k1, p, first_cp(a), first_cp(b - 1) + p + 1,
                                    first_cp(w0), first_cp(w1 - 1) + p + 1))
        else:
            pieces.append(AxisPiece(a, b, w0, w1, k0, k1, p))
        a = b
    return pieces


# ---------------------------------------------------------------------------
# Tensor helpers (plain numpy; grid axis a <-> numpy axis d-1-a)
# ---------------------------------------------------------------------------


def _np_axis(a: int, d: int) -> int:
    return d - 1 - a


def apply_along_axis(T: np.ndarray, mat: np.ndarray, a: int) -> np.ndarray:
    """Contract grid axis a of tensor T with matrix ``mat``: out_i = sum_j mat[i, j] T_j."""
    d = T.ndim
    ax = _np_axis(a, d)
    out = np.tensordot(mat, T, axes=([1], [ax]))  # new axis first
    return np.moveaxis(out, 0, ax)


def box(T: np.ndarray, ranges: Sequence[range]) -> np.ndarray:
    """Sub-array of T selected by one index range per grid axis."""
    d = T.ndim
    sl = [None] * d
    for a, r in enumerate(ranges):
        sl[_np_axis(a, d)] = slice(r.start, r.stop)
    return T[tuple(sl)]


def _box_slices(ranges: Sequence[range], d: int):
    sl = [None] * d
    for a, r in enumerate(ranges):
        sl[_np_axis(a, d)] = slice(r.start, r.stop)
    return tuple(sl)


# ---------------------------------------------------------------------------
# Sec. 2.1 / 2.3.1: separable least squares through the normal equations
# ---------------------------------------------------------------------------


class NotSPDError(RuntimeError):
    pass


def cholesky_solve(A: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve A X = rhs with a Cholesky factorisation (Sec. 2.3.1)."""
    try:
        c = scipy.linalg.cho_factor(A, lower=True, check_finite=True)
    except np.linalg.LinAlgError as e:  # not positive definite
        raise NotSPDError(str(e)) from e
    return scipy.linalg.cho_solve(c, rhs)


def separable_lsq(Qbox: np.ndarray, mats: Sequence[np.ndarray]) -> np.ndarray:
    """argmin_P || Q - (N_{d-1} x ... x N_0) P ||_2 for a tensor-grid box.

    The normal matrix of the Kronecker collocation matrix is the Kronecker
    product of the per-axis Gram matrices N_a^T N_a, so the normal equations
    (Eq. minimization-problem) are solved by projecting every axis with N_a^T
    and then applying (N_a^T N_a)^{-1} on every axis, axis 0 first.
    """
    T = Qbox
    for a, N in enumerate(mats):
        T = apply_along_axis(T, N.T, a)
    for a, N in enumerate(mats):
        A = N.T @ N
        T = apply_along_axis(T, cholesky_solve(A, np.eye(A.shape[0])), a)
    return T


def decode_box(P: np.ndarray, mats: Sequence[np.ndarray]) -> np.ndarray:
    """Tensor-product decode R P = (N_{d-1} x ... x N_0) P (Algorithm 1 error step)."""
    T = P
    for a, N in enumerate(mats):
        T = apply_along_axis(T, N, a)
    return T


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------


@dataclass
class Problem:
    """A gridded MFA problem in the adopted reading.

    npts[a], nspans[a], cores[a] (list of core span counts), delta[a] per grid
    axis a = 0..d-1, one degree p for all axes.  ``clamped``: interface knots
    repeated p times (Sec. 2.2 / 3.1.1 clamped variant) instead of floating.
    ``weights``: None (B-splines, W = 1) or one array of control-point weights
    per axis (separable NURBS weights, Eq. nurbs-basis).
    """

    p: int
    npts: List[int]
    nspans: List[int]
    cores: List[List[int]]
    delta: List[int]
    clamped: bool = False
    weights: Optional[List[np.ndarray]] = None

    @property
    def d(self) -> int:
        return len(self.npts)

    def knot_ints(self, a: int) -> List[int]:
        return knot_ints(self.nspans[a], self.p, self.cores[a] if self.clamped else None)

    def ncp(self) -> List[int]:
        return [len(self.knot_ints(a)) - self.p - 1 for a in range(self.d)]

    def knots(self, a: int) -> np.ndarray:
        return np.array(self.knot_ints(a), dtype=np.float64) / self.nspans[a]

    def params(self, a: int) -> np.ndarray:
        return grid_params(self.npts[a])

    def basis_at(self, a: int, u, deriv: int = 0, side: str = "right") -> np.ndarray:
        """Basis rows of axis a (rational when weights are given) at parameters u."""
        if self.weights is None:
            return basis_matrix(self.knots(a), self.p, u, deriv, side)
        return rational_basis(self.knots(a), self.p, self.weights[a], u, deriv, side)

    def basis(self, a: int) -> np.ndarray:
        return self.basis_at(a, self.params(a))

    def pieces(self, a: int) -> List[AxisPiece]:
        return axis_pieces(self.npts[a], self.nspans[a], self.p, self.cores[a], self.delta[a], self.clamped)

    def subdomains(self):
        """All subdomains as tuples of AxisPiece, axis 0 varying fastest."""
        per_axis = [self.pieces(a) for a in range(self.d)]
        out = []
        for idx in np.ndindex(*[len(x) for x in reversed(per_axis)]):
            s = tuple(per_axis[a][idx[self.d - 1 - a]] for a in range(self.d))
            out.append(s)
        return out


def make_problem(p, npts, nspans, nsub, delta, cores=None, clamped=False, weights=None) -> Problem:
    """A decomposed fit (Sec. 2.2): degree p, grid points and global knot spans
    per axis, subdomains per axis (cores split evenly unless given), and the
    overlap delta in knot spans (one value or one per axis).  ``clamped``
    selects clamped interface knots; ``weights`` per-axis NURBS weights."""
    d = len(npts)
    if cores is None:
        cores = [even_cores(nspans[a], nsub[a]) for a in range(d)]
    if isinstance(delta, int):
        delta = [delta] * d
    prob = Problem(p, list(npts), list(nspans), [list(c) for c in cores], list(delta), bool(clamped))
    if weights is not None:
        prob.weights = [np.asarray(w, np.float64) for w in weights]
        for a in range(d):
            assert prob.weights[a].shape == (prob.ncp()[a],) and (prob.weights[a] > 0).all()
    return prob


# ---------------------------------------------------------------------------
# The plain definition: global LSQ fit (N = 1)
# ---------------------------------------------------------------------------


def global_fit(prob: Problem, Q: np.ndarray) -> np.ndarray:
    """argmin_P ||Q - R P|| over the whole grid (Eq. minimization-problem, N = 1)."""
    return separable_lsq(np.asarray(Q, np.float64), [prob.basis(a) for a in range(prob.d)])


def decode_grid(prob: Problem, P: np.ndarray) -> np.ndarray:
    """Decode the global control points on the full data grid."""
    return decode_box(P, [prob.basis(a) for a in range(prob.d)])


# ---------------------------------------------------------------------------
# Sec. 2.3 / Algorithm 1: overlapping additive Schwarz
# ---------------------------------------------------------------------------


@dataclass
class SchwarzState:
    P: np.ndarray                      # current global iterate P^k
    copies: list                       # per-subdomain owned copies (arrays over U_s)
    frames: list                       # per-subdomain L_s arrays used in the last solve
    k: int = 0
    history: list = field(default_factory=list)


def _local_mats(prob: Problem, s, Nglob, cols: str):
    """Per-axis collocation matrices of subdomain s (Sec. 2.2): its window's
    data rows against its local control points L (cols = "L") or its owned
    ones U (cols = "U"), cut from the global basis matrices."""
    mats = []
    for a, pc in enumerate(s):
        rows = pc.pts
        cr = pc.L if cols == "L" else pc.U
        mats.append(Nglob[a][rows.start:rows.stop, cr.start:cr.stop])
    return mats


def greville_owner(prob: Problem, a: int) -> np.ndarray:
    """Owner-takes update (the restricted additive Schwarz variant of Sec. 2.3):
    along axis a, the subdomain whose core span range [a_s, b_s) holds the
    Greville abscissa xi_g = (t_{g+1} + ... + t_{g+p}) / p of control point g
    (the last core also holds xi = 1).  Decided exactly: with knots
    t_i = k_i / nspans, xi_g * nspans * p is the integer sum of the k_i."""
    p = prob.p
    k = prob.knot_ints(a)  # t_i = k[i] / nspans
    n = len(k) - p - 1
    pcs = prob.pieces(a)
    own = np.empty(n, dtype=np.int64)
    for g in range(n):
        S = sum(k[g + 1:g + p + 1]) if p > 0 else k[g] + k[g + 1]
        den = p if p > 0 else 2
        own[g] = -1
        for i, pc in enumerate(pcs):
            last = i == len(pcs) - 1
            if pc.a * den <= S and (S < pc.b * den or (last and S <= pc.b * den)):
                own[g] = i
                break
        if own[g] < 0:
            raise ValueError("Greville abscissa outside every core")
    return own


def average_copies(prob: Problem, subs, copies, update: str = "average") -> tuple:
    """Update of the global control points from the owned copies.

    update="average": uniformly weighted average of every owned copy,
    w = 1/n_s (Sec. 2.3.2).  update="owner": every control point takes the
    copy of the subdomain owning its Greville abscissa (greville_owner),
    axis by axis in the tensor product.

    Returns (P, spread) where spread[g] = max copy - min copy of CP g."""
    if update == "owner":
        P, spread = average_copies(prob, subs, copies, "average")
        own = [greville_owner(prob, a) for a in range(prob.d)]
        pieces = [prob.pieces(a) for a in range(prob.d)]
        P = np.full(P.shape, np.nan)
        for s, c in zip(subs, copies):
            masks = []
            for a in range(prob.d):
                ia = pieces[a].index(s[a])
                masks.append(own[a][list(s[a].U)] == ia)
            M = masks[0]
            for a in range(1, prob.d):
                M = np.multiply.outer(masks[a], M)  # numpy axis order: last grid axis first
            sl = _box_slices([pc.U for pc in s], prob.d)
            view = P[sl]
            view[M] = c[M]
        if np.isnan(P).any():
            raise ValueError("a control point has no Greville owner among its owning subdomains")
        return P, spread
    shape = tuple(reversed(prob.ncp()))
    acc = np.zeros(shape)
    cnt = np.zeros(shape)
    hi = np.full(shape, -np.inf)
    lo = np.full(shape, np.inf)
    for s, c in zip(subs, copies):
        sl = _box_slices([pc.U for pc in s], prob.d)
        acc[sl] += c
        cnt[sl] += 1
        hi[sl] = np.maximum(hi[sl], c)
        lo[sl] = np.minimum(lo[sl], c)
    if np.any(cnt == 0):
        raise ValueError("a control point is owned by no subdomain")
    return acc / cnt, hi - lo


def schwarz_initial(prob: Problem, Q: np.ndarray, update: str = "average") -> SchwarzState:
    """Iteration 0 of Algorithm 1: every subdomain solves the unconstrained
    local LSQ on its window data with all of L_s free (Eq. minimization-problem);
    the owned part U_s of each local solution is kept and averaged."""
    Q = np.asarray(Q, np.float64)
    Nglob = [prob.basis(a) for a in range(prob.d)]
    subs = prob.subdomains()
    copies, frames = [], []
    for s in subs:
        mats = _local_mats(prob, s, Nglob, "L")
        PL = separable_lsq(box(Q, [pc.pts for pc in s]), mats)
        frames.append(PL)
        u_in_l = [range(pc.oU, pc.oU + len(pc.U)) for pc in s]
        copies.append(box(PL, u_in_l).copy())
    P, spread = average_copies(prob, subs, copies, update)
    st = SchwarzState(P=P, copies=copies, frames=frames, k=0)
    st.history.append({"k": 0, "spread": float(spread.max(initial=0.0))})
    return st


def schwarz_step(prob: Problem, Q: np.ndarray, st: SchwarzState, update: str = "average") -> SchwarzState:
    """One outer iteration k >= 1 of Algorithm 1.

    Exchange: each subdomain reads its frame F_s = L_s minus U_s from the
    lagged global iterate P^{k-1} (the dequeued constraints P_i(Delta u delta)).
    Constrain: the frame is held fixed, its decoded contribution is moved to
    the right-hand side, and the owned points U_s are re-solved by LSQ on the
    window data -- the Schur-complement decoupling with lagged neighbour
    values (Sec. 2.2, Eq. global-system; jump terms of Eq. nonlinear-residuals
    driven to zero at the fixed point).
    Update: P^k averages all owned copies with w = 1/n_s (Sec. 2.3.2).
    """
    Q = np.asarray(Q, np.float64)
    Nglob = [prob.basis(a) for a in range(prob.d)]
    subs = prob.subdomains()
    copies, frames = [], []
    for s in subs:
        Lr = [pc.L for pc in s]
        PF = box(st.P, Lr).copy()
        u_in_l = [range(pc.oU, pc.oU + len(pc.U)) for pc in s]
        PF[_box_slices(u_in_l, prob.d)] = 0.0
        matsL = _local_mats(prob, s, Nglob, "L")
        R = box(Q, [pc.pts for pc in s]) - decode_box(PF, matsL)
        PU = separable_lsq(R, _local_mats(prob, s, Nglob, "U"))
        full = PF.copy()
        full[_box_slices(u_in_l, prob.d)] = PU
        frames.append(full)
        copies.append(PU)
    P, spread = average_copies(prob, subs, copies, update)
    dP = float(np.max(np.abs(P - st.P)))
    pmax = float(np.max(np.abs(P)))
    new = SchwarzState(P=P, copies=copies, frames=frames, k=st.k + 1, history=list(st.history))
    new.history.append({"k": new.k, "dP_rel": dP / pmax if pmax > 0 else 0.0,
                        "spread": float(spread.max(initial=0.0))})
    return new


def residual_stats(prob: Problem, Q: np.ndarray, P: np.ndarray) -> dict:
    """Decoded error E = Q - R P over the full grid: RMS and max |E|."""
    E = np.asarray(Q, np.float64) - decode_grid(prob, P)
    return {"rms": float(np.sqrt(np.mean(E * E))), "max": float(np.max(np.abs(E)))}


def schwarz_solve(prob: Problem, Q: np.ndarray, max_iters: int = 200, tol_dP: float = 0.0,
                  tol_rms_stall: float = 0.0, keep_iterates: bool = False, update: str = "average") -> dict:
    """Algorithm 1 to convergence.

    Stops after iteration k >= 1 when dP_rel = max|P^k - P^{k-1}| / max|P^k|
    <= tol_dP, or (if tol_rms_stall > 0) when the decoded RMS changes by at
    most tol_rms_stall * RMS_k, or at max_iters.
    """
    st = schwarz_initial(prob, Q, update)
    iterates = [st.P.copy()] if keep_iterates else None
    rms_prev = residual_stats(prob, Q, st.P)["rms"] if tol_rms_stall > 0 else None
    converged = False
    while st.k < max_iters:
        st = schwarz_step(prob, Q, st, update)
        if keep_iterates:
            iterates.append(st.P.copy())
        h = st.history[-1]
        if h["dP_rel"] <= tol_dP:
            converged = True
            break
        if tol_rms_stall > 0:
            rms = residual_stats(prob, Q, st.P)["rms"]
            h["rms"] = rms
            if abs(rms - rms_prev) <= tol_rms_stall * rms:
                converged = True
                break
            rms_prev = rms
    return {"P": st.P, "state": st, "iters": st.k, "converged": converged,
            "iterates": iterates, "history": st.history}


# ---------------------------------------------------------------------------
# Continuity diagnostics (Sec. 2.2: C^0 .. C^{p-1} at interfaces)
# ---------------------------------------------------------------------------


def interface_jumps(prob: Problem, st: SchwarzState, max_order: Optional[int] = None) -> np.ndarray:
    """Jumps of derivative orders 0..max_order between the local splines of
    neighbouring subdomains at every interface (Sec. 2.2: C^0 .. C^{p-1};
    Algorithm 1 "check convergence metrics").

    The local spline of subdomain s is the one it solved last: its L box of
    control points, the owned copy plus the frame it held (``st.frames``).  At
    an interface between pieces i and i+1 along axis a (breakpoint
    tau = b_i / nspans_a) the left subdomain is evaluated as a left limit and
    the right one as a right limit, for every pair of subdomains that differ
    only in their piece along a.  Along the other axes the samples are the
    data points of the pair's common core (closed core interval).  Order r is
    the r-th derivative along a with respect to the knot coordinate
    x = u * nspans_a (span units, so every order has the scale of the data).

    Returns an array [n_interface_pairs, max_order + 1] of maxima over each
    pair's samples, pairs ordered by axis, then by subdomain index."""
    p, d = prob.p, prob.d
    if max_order is None:
        max_order = p
    subs = prob.subdomains()
    pieces = [prob.pieces(a) for a in range(d)]
    Nfull = [prob.basis(a) for a in range(d)]
    index = {tuple(pieces[a].index(s[a]) for a in range(d)): i for i, s in enumerate(subs)}
    out = []
    for a in range(d):
        ns = prob.nspans[a]
        for key, i in sorted(index.items(), key=lambda kv: (kv[1])):
            if key[a] + 1 >= len(pieces[a]):
                continue
            nkey = list(key)
            nkey[a] += 1
            j = index[tuple(nkey)]
            sL, sR = subs[i], subs[j]
            tau = sL[a].b / ns
            row = []
            for r in range(max_order + 1):
                vals = []
                for s, X, side in ((sL, st.frames[i], "left"), (sR, st.frames[j], "right")):
                    mats = []
                    for b in range(d):
                        Lr = s[b].L
                        if b == a:
                            D = prob.basis_at(a, [tau], r, side) / ns ** r
                            mats.append(D[:, Lr.start:Lr.stop])
                        else:
                            M = prob.npts[b]
                            lo, hi = s[b].a, s[b].b
                            ks = [k for k in range(M)
                                  if M == 1 or lo * (M - 1) <= k * prob.nspans[b] <= hi * (M - 1)]
                            mats.append(Nfull[b][ks][:, Lr.start:Lr.stop])
                    vals.append(decode_box(X, mats))
                row.append(float(np.max(np.abs(vals[0] - vals[1]))))
            out.append(row)
    return np.array(out).reshape(-1, max_order + 1)


def global_jumps(prob: Problem, P: np.ndarray, max_order: Optional[int] = None) -> np.ndarray:
    """Jumps of derivative orders 0..max_order of the global spline (control
    points P) across every interface breakpoint, as one-sided limits (Sec. 2.2:
    floating interface knots keep the global spline C^{p-1}, clamped interface
    knots only C^0).  Samples along the other axes are all data points; order
    r is in span units as in interface_jumps.  Returns [n_interfaces_total,
    max_order + 1]."""
    p, d = prob.p, prob.d
    if max_order is None:
        max_order = p
    Nfull = [prob.basis(a) for a in range(d)]
    out = []
    for a in range(d):
        ns = prob.nspans[a]
        for pc in prob.pieces(a)[:-1]:
            tau = pc.b / ns
            row = []
            for r in range(max_order + 1):
                v = []
                for side in ("left", "right"):
                    mats = [Nfull[b] if b != a else prob.basis_at(a, [tau], r, side) / ns ** r for b in range(d)]
                    v.append(decode_box(P, mats))
                row.append(float(np.max(np.abs(v[0] - v[1]))))
            out.append(row)
    return np.array(out).reshape(-1, max_order + 1)


def scattered_decode(prob: Problem, P: np.ndarray, u: np.ndarray, deriv=None) -> np.ndarray:
    """Evaluate the global tensor spline (or a mixed partial derivative with
    per-axis orders ``deriv``) at parameter points u[k, a] in [0,1]^d, one point
    at a time through dense basis rows."""
    d = prob.d
    u = np.atleast_2d(np.asarray(u, np.float64))
    deriv = [0] * d if deriv is None else list(deriv)
    out = np.empty(len(u))
    for k in range(len(u)):
        T = P
        for a in range(d):
            row = prob.basis_at(a, [u[k, a]], deriv[a])  # (1, n_a)
            T = apply_along_axis(T, row, a)
        out[k] = float(np.asarray(T).reshape(-1)[0])
    return out
