"""Write the stored expected values under tests/golden/ (calls only the oracle).

fig1_oracle_n1e5.json: the FP64 oracle's estimate, standard error and mean |f|
for the paper's 100 harmonics of Eq. 1 (Sec. "Test on GPUs": a_n = b_n = 1,
box [0,1]^4, k_n = (n+50)/(2 pi) (1,1,1,1)) at 10^5 samples each, Philox key 0,
stream id n-1.  The paper prints no values for this test (its Fig. 1 is a plot
against the analytic curve), so the file pins the oracle against regressions and
lets GPU tests compare without re-running the oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2104_10073_gb300 import workloads as W  # noqa: E402


def main():
    tab = W.harmonic_fig1(10**5)
    res, _ = oracle.integrate(tab)
    out = {
        "source": "oracle/zmc_oracle.c via tests/golden/make_golden.py",
        "workload": "paper Eq. 1 / Fig. 1 harmonics, n=1..100, N=1e5, key 0, stream n-1",
        "estimate": [float(v).hex() for v in res["estimate"]],
        "stderr": [float(v).hex() for v in res["stderr"]],
        "mean_abs": [float(v).hex() for v in res["mean_abs"]],
    }
    with open(os.path.join(HERE, "fig1_oracle_n1e5.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
