"""The host estimate of cond(N^T N) that chooses which FP32 batch instances
get a refinement step (mfa_gram_condition, no GPU): checked against numpy's
exact 2-norm condition number of the dense normal matrix of an independent
basis (scipy's B-spline design matrix on the same clamped uniform knots and
points)."""
import numpy as np
import pytest

from paper_2210_06528_gb300 import mfa


def _dense_cond(M, ns, p):
    BSpline = pytest.importorskip("scipy.interpolate").BSpline
    t = np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, ns + 1), np.ones(p)])
    N = BSpline.design_matrix(np.linspace(0.0, 1.0, M), t, p).toarray()
    return np.linalg.cond(N.T @ N)


@pytest.mark.parametrize("M,ns,p", [(16, 1, 3), (40, 8, 2), (64, 13, 3), (128, 28, 4), (200, 45, 5), (100, 20, 1),
                                    (33, 31, 2), (512, 125, 3), (90, 10, 7)])
def test_estimate_matches_the_dense_condition_number(M, ns, p):
    est = mfa.mfa_gram_condition(M, ns, p)
    exact = _dense_cond(M, ns, p)
    assert abs(est - exact) <= 0.03 * exact, (est, exact)


def test_rank_deficient_normal_matrix_is_flagged():
    # more control points (ns + p = 9) than points: N^T N is singular
    assert mfa.mfa_gram_condition(6, 6, 3) >= 1e300


@pytest.mark.parametrize("args", [(0, 4, 3), (64, 0, 3), (64, 4, 0), (64, 4, 8)])
def test_arguments_out_of_range_are_refused(args):
    with pytest.raises(mfa.MFAError) as e:
        mfa.mfa_gram_condition(*args)
    assert e.value.code == mfa.MFA_ERR_ARG


def test_rule_on_the_batched_workload():
    """2^-24 x the product of sqrt(cond) over an instance's axes above 2e-6
    marks 2514 of the 4096 instances of the batched workload for a
    refinement step (the count the GPU batch reports): every 3-D instance of
    degree >= 4 and 2-D instance of degree 5, none of degree 2 in 3-D or
    degree <= 3 in 2-D; 3-D degree 3 and 2-D degree 4 depend on the shape."""
    from paper_2210_06528_gb300 import inputs
    specs, _ = inputs.batch_instances(4096, seed=0)
    cache = {}
    refined = 0
    kinds = set()
    for sp in specs:
        g = 2.0 ** -24
        for M, ns in zip(sp["npts"], sp["nspans"]):
            key = (M, ns, sp["degree"])
            if key not in cache:
                cache[key] = mfa.mfa_gram_condition(M, ns, sp["degree"])
            g *= np.sqrt(cache[key])
        refined += g > 2e-6
        kinds.add((sp["dim"], sp["degree"], bool(g > 2e-6)))
    assert refined == 2514
    for d, p, r in kinds:
        if (d == 3 and p >= 4) or (d == 2 and p == 5):
            assert r, (d, p)
        if (d == 3 and p == 2) or (d == 2 and p <= 3):
            assert not r, (d, p)
