"""Fixtures of numbers the paper prints (tests/golden/, each file citing its
passage), checked against the oracle's layout on the CPU.

The paper prints no worked example of a fit. What it does print is the
arithmetic of two compression ratios, total input points over total control
points. Both count the global control points per axis as (subdomains per
axis) x (control points per subdomain). That fixes how "n control points per
subdomain" is read: n core knot spans per subdomain, the global knot vector
then holding N n spans (and N n + p control points, the p end ones being
what the paper's count leaves out). The other reading, n local control
points per subdomain (n - p core spans), gives a ratio far from the printed
one and is rejected here.
"""
import os

import numpy as np
import pytest

from oracle import mfa_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = [float(x) for x in rest]
    return vals


@pytest.mark.parametrize("name,digits", [("s3d_compression_ratio.txt", 1),
                                         ("nek5000_slice_compression_ratio.txt", 0)])
def test_printed_compression_ratio_fixes_the_control_point_reading(name, digits):
    g = read_fixture(name)
    grid = [int(x) for x in g["grid"]]
    N = int(g["subdomains_per_axis"][0])
    n = int(g["n_per_subdomain"][0])
    p = int(g["degree"][0])
    delta = int(g["overlap"][0])
    printed = g["compression_ratio_printed"][0]
    d = len(grid)
    # reading: n core spans per subdomain, N n spans on the global knot vector
    prob = O.make_problem(p, grid, [N * n] * d, [N] * d, delta)
    for a in range(d):
        pcs = prob.pieces(a)
        assert len(pcs) == N
        assert all(pc.b - pc.a == n for pc in pcs)
        assert prob.ncp()[a] - p == N * n
    # the paper's arithmetic on the oracle's layout reproduces the printed ratio
    eta_paper = np.prod(grid) / np.prod([prob.ncp()[a] - p for a in range(d)])
    assert round(eta_paper, digits) == printed
    # counting the p end control points too changes it by a few per cent only
    eta_all = np.prod(grid) / np.prod(prob.ncp())
    assert abs(eta_all - printed) / printed < 0.15
    # n local control points per subdomain (n - p core spans) misses the printed value
    eta_local = np.prod(grid) / np.prod([N * (n - p) + p] * d)
    assert abs(eta_local - printed) / printed > 0.25
