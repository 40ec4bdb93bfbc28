"""Serving runtime: continuous batching of encode requests and decode queries.

Every fit and every decoded value is the same whether a request runs alone or
in a mix with others in flight (each instance is computed independently of
the rest of its batch), admission keeps the reserved memory within the
budget, and a query of a released model fails cleanly."""
import numpy as np
import pytest

from mfa_cases import TOL_FP64, rel_diff
from oracle import mfa_oracle as O
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu


def _workload(seed, count=8):
    specs, data = inputs.batch_instances(count, seed=seed, size2=(24, 90), size3=(12, 28), degrees=(3, 3),
                                         dims=(2, 3))
    payloads = [data[sp["q_offset"]:sp["q_offset"] + int(np.prod(sp["npts"]))].copy() for sp in specs]
    rng = np.random.default_rng(seed)
    queries = []
    for i in range(count):
        for _ in range(2):
            n = int(rng.integers(1, 3000))
            queries.append((i, rng.uniform(0, 1, size=(n, 3))))
    return specs, payloads, queries


def _run(srv, specs, payloads, queries, alone):
    models, ctrl, vals = [], [], []
    if alone:
        for sp, q in zip(specs, payloads):
            rid = srv.encode(sp, q)
            rc, _ = srv.wait(rid)
            assert rc == mfa.MFA_OK
            models.append(rid)
        outs = []
        for i, u in queries:
            out = np.empty(len(u))
            rc, _ = srv.wait(srv.decode(models[i], u, out))
            assert rc == mfa.MFA_OK
            outs.append(out)
    else:
        models = [srv.encode(sp, q) for sp, q in zip(specs, payloads)]
        outs = [np.empty(len(u)) for _, u in queries]
        rids = [srv.decode(models[i], u, o) for (i, u), o in zip(queries, outs)]  # before the fits finish
        for rid in models + rids:
            rc, _ = srv.wait(rid, 120.0)
            assert rc == mfa.MFA_OK
    for m in models:
        ctrl.append(srv.ctrl(m))
    return models, ctrl, outs


def test_results_alone_equal_results_in_the_mix():
    specs, payloads, queries = _workload(21)
    srv = mfa.Server(0, workers=3, mem_budget=4 << 30)
    try:
        m1, c1, v1 = _run(srv, specs, payloads, queries, alone=True)
        m2, c2, v2 = _run(srv, specs, payloads, queries, alone=False)
        for a, b in zip(c1, c2):
            assert np.array_equal(a, b)
        for a, b in zip(v1, v2):
            assert np.array_equal(a, b)
        st = srv.stats()
        assert st["resident_models"] == 2 * len(specs)
        # parity of the served fit with the oracle's global fit
        for i in (0, 3):
            sp = specs[i]
            Q = payloads[i].astype(np.float64).reshape(tuple(reversed(sp["npts"])))
            prob = O.make_problem(sp["degree"], list(sp["npts"]), list(sp["nspans"]), [1] * sp["dim"], 0)
            assert rel_diff(c1[i], O.global_fit(prob, Q).ravel()) <= TOL_FP64
        for m in m1 + m2:
            srv.release(m)
        assert srv.stats()["reserved"] == 0
    finally:
        srv.close()


def test_admission_under_a_tight_budget():
    """A budget that fits a few requests at a time: everything still
    completes in order of admission and the reservation never exceeds it."""
    specs, payloads, queries = _workload(5, count=10)
    budget = 24 << 20
    srv = mfa.Server(0, workers=2, mem_budget=budget)
    try:
        ids = [srv.encode(sp, q) for sp, q in zip(specs, payloads)]
        infos = []
        for rid in ids:
            rc, info = srv.wait(rid, 120.0)
            assert rc == mfa.MFA_OK
            infos.append(info)
        st = srv.stats()
        assert st["peak_reserved"] <= budget
        assert all(infos[k]["t_admit"] <= infos[k + 1]["t_admit"] for k in range(len(infos) - 1))
        for rid in ids:
            srv.release(rid)
        assert srv.stats()["reserved"] == 0
        with pytest.raises(mfa.MFAError) as ei:
            srv.encode(dict(specs[0], npts=[4000, 4000], nspans=[900, 900], dim=2), np.zeros(16_000_000, np.float32))
        assert ei.value.code == mfa.MFA_ERR_OOM
    finally:
        srv.close()


def test_query_of_a_released_model_fails():
    specs, payloads, queries = _workload(9, count=2)
    srv = mfa.Server(0, workers=1, mem_budget=1 << 30)
    try:
        m = srv.encode(specs[0], payloads[0])
        assert srv.wait(m)[0] == mfa.MFA_OK
        srv.release(m)
        with pytest.raises(mfa.MFAError):
            srv.decode(m, np.zeros((4, 3)), np.empty(4))
    finally:
        srv.close()


def _run_prec(srv, specs, payloads, queries, alone, precision):
    models, outs = [], []
    if alone:
        for sp, q in zip(specs, payloads):
            rid = srv.encode(sp, q, precision)
            rc, _ = srv.wait(rid)
            assert rc == mfa.MFA_OK
            models.append(rid)
        for i, u in queries:
            out = np.empty(len(u))
            rc, _ = srv.wait(srv.decode(models[i], u, out))
            assert rc == mfa.MFA_OK
            outs.append(out)
    else:
        models = [srv.encode(sp, q, precision) for sp, q in zip(specs, payloads)]
        outs = [np.empty(len(u)) for _, u in queries]
        rids = [srv.decode(models[i], u, o) for (i, u), o in zip(queries, outs)]
        for rid in models + rids:
            rc, _ = srv.wait(rid, 120.0)
            assert rc == mfa.MFA_OK
    return models, [srv.ctrl(m) for m in models], outs


def test_fp32_encodes_alone_equal_the_mix_and_meet_the_bar():
    """Served encodes in FP32 data-pass precision: the same control points
    and decoded values alone and in the mix, and the decoded values within
    1e-5 of the data range of the oracle's global fit decoded at the same
    points."""
    specs, payloads, queries = _workload(33)
    srv = mfa.Server(0, workers=3, mem_budget=4 << 30)
    try:
        m1, c1, v1 = _run_prec(srv, specs, payloads, queries, True, mfa.MFA_PREC_FP32)
        m2, c2, v2 = _run_prec(srv, specs, payloads, queries, False, mfa.MFA_PREC_FP32)
        for a, b in zip(c1, c2):
            assert np.array_equal(a, b)
        for a, b in zip(v1, v2):
            assert np.array_equal(a, b)
        for qi, (i, u) in enumerate(queries):
            sp = specs[i]
            Q = payloads[i].astype(np.float64).reshape(tuple(reversed(sp["npts"])))
            prob = O.make_problem(sp["degree"], list(sp["npts"]), list(sp["nspans"]), [1] * sp["dim"], 0)
            want = O.scattered_decode(prob, O.global_fit(prob, Q), u[:, :sp["dim"]])
            rng = float(Q.max() - Q.min())
            assert np.abs(v1[qi] - want).max() <= 1e-5 * rng, (qi, sp)
        for m in m1 + m2:
            srv.release(m)
    finally:
        srv.close()


_FIRST_ENCODES = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2210_06528_gb300 import inputs, mfa
specs, data = inputs.batch_instances(12, seed=41, size2=(64, 400), size3=(32, 160), degrees=(2, 5))
srv = mfa.Server(0, workers=3, mem_budget=16 << 30, max_batch=1)
try:
    rids = [srv.encode(sp, data[sp["q_offset"]:sp["q_offset"] + int(np.prod(sp["npts"]))], mfa.MFA_PREC_FP32)
            for sp in specs]
    codes = [srv.wait(r, 300.0)[0] for r in rids]
finally:
    srv.close()
print(codes)
sys.exit(0 if all(c == mfa.MFA_OK for c in codes) else 1)
"""


def test_first_fp32_encodes_of_different_sizes_at_once():
    """A fresh process whose first launches are served FP32 encodes of
    different sizes on three workers at once, one instance per job: every
    launch raises its kernel's shared-memory limit as needed while other
    workers launch the same kernels with other sizes, and every encode
    succeeds."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_ENCODES, root], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
