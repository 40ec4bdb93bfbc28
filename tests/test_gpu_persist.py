"""Persistence of fitted models: a saved and reloaded model holds the same
control points, decodes the same values and (with its Schwarz state) iterates
on exactly as the original would."""
import os

import numpy as np
import pytest

from mfa_cases import GpuFit
from paper_2210_06528_gb300 import inputs, mfa

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [mfa.MFA_PREC_FP64, mfa.MFA_PREC_MIXED])
def test_save_load_roundtrip_and_continue(tmp_path, precision):
    Q = inputs.gauss_3d((40, 36, 34), seed=8, dtype=np.float32)
    g = GpuFit(Q, 3, [12, 11, 10], [2, 2, 2], 2, precision=precision)
    try:
        g.model.set_update_rule(mfa.MFA_UPDATE_OWNER)
        g.iterate(2, 0.0)
        path = str(tmp_path / "model.mfa")
        g.model.save(path, state=True)
        m2 = g.handle.load(path)
        assert np.array_equal(m2.ctrl(), g.ctrl())
        D1 = g.decode_grid()
        D2 = np.empty(Q.shape)
        m2.decode_grid(D2)
        assert np.array_equal(D1, D2)
        rc1, rep1 = g.iterate(3, 0.0)
        rc2, rep2 = m2.iterate(3, 0.0)
        assert rep1.iters == rep2.iters == 5
        assert np.array_equal(m2.ctrl(), g.ctrl())
        r1, r2 = g.residual(), m2.residual(g.q)
        assert r1.rms_decoded == r2.rms_decoded
        m2.free()
    finally:
        g.close()


def test_stateless_load_decodes_but_does_not_iterate(tmp_path):
    Q = inputs.gauss_3d((30, 28, 26), seed=2, dtype=np.float32)
    g = GpuFit(Q, 3, [9, 8, 7], [2, 1, 2], 1)
    try:
        g.iterate(3, 0.0)
        path = str(tmp_path / "m.mfa")
        g.model.save(path)
        m2 = g.handle.load(path)
        D = np.empty(Q.shape)
        m2.decode_grid(D)
        assert np.array_equal(D, g.decode_grid())
        with pytest.raises(mfa.MFAError) as ei:
            m2.iterate(1, 0.0)
        assert ei.value.code == mfa.MFA_ERR_ARG
        m2.free()
        # a damaged file is refused
        with open(path, "r+b") as f:
            f.write(b"XXXX")
        with pytest.raises(mfa.MFAError) as ei:
            g.handle.load(path)
        assert ei.value.code == mfa.MFA_ERR_IO
        with pytest.raises(mfa.MFAError) as ei:
            g.handle.load(os.path.join(str(tmp_path), "missing.mfa"))
        assert ei.value.code == mfa.MFA_ERR_IO
    finally:
        g.close()
