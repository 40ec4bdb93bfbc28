"""Write workload_rms.json: the FP64 oracle's Schwarz-converged fit of the
1-D and 2-D workloads (iterations, decoded RMS and max |error|), the values
the GPU runs of the same workloads are reported beside.

Calls only the oracle and the seeded input generators:

  python tests/golden/make_workload_rms.py

  * 1-D: 1024 points of sin(x)/x on [-4 pi, 4 pi] (Sec. 3.1), p = 3, 128
    uniform spans in 4 subdomains, overlap 2, FP64, Schwarz to
    dP_rel <= 1e-10 (Algorithm 1 with the control-point change as the
    convergence metric).
  * 2-D: 1024^2 sinc(x) sinc(y) on [-4 pi, 4 pi]^2 + N(0, 1e-3) (Sec. 3.2,
    seed 0, stored as FP32), p = 3, 256 spans per axis in 4x4 subdomains,
    overlap 2, Schwarz to decoded-residual stall |RMS_k - RMS_{k-1}| <=
    1e-6 RMS_k.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mfa_oracle as O  # noqa: E402
from paper_2210_06528_gb300 import inputs  # noqa: E402


def run(Q, p, nspans, nsub, delta, max_iters, tol_dP, tol_rms_stall):
    prob = O.make_problem(p, list(Q.shape[::-1]), list(nspans), list(nsub), delta)
    res = O.schwarz_solve(prob, Q, max_iters=max_iters, tol_dP=tol_dP, tol_rms_stall=tol_rms_stall)
    st = O.residual_stats(prob, Q, res["P"])
    return {"iters": int(res["iters"]), "converged": bool(res["converged"]), "rms": float(st["rms"]),
            "max": float(st["max"])}


def main():
    out = {}
    out["1d"] = dict(run(inputs.sinc_1d(1024).astype(np.float64), 3, [128], [4], 2, 200, 1e-10, 0.0),
                     workload="1d_1024_sinc_p3_4sub_32spans_overlap2_fp64", stop="dP_rel <= 1e-10")
    q2 = inputs.sinc_2d(1024, noise=1e-3, seed=0, dtype=np.float32).astype(np.float64)
    out["2d"] = dict(run(q2, 3, [256, 256], [4, 4], 2, 50, 0.0, 1e-6),
                     workload="2d_1024^2_sinc_noise1e-3_p3_4x4sub_64spans_overlap2",
                     stop="|RMS_k - RMS_{k-1}| <= 1e-6 RMS_k")
    with open(os.path.join(HERE, "workload_rms.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
