"""Physics validation of the whole step against a value the paper prints.

Table 2, case 1 (tests/golden/table2_case1.json): Ra = 1e4, Pr = 0.7,
gamma = 5/3, eps = 0.1, D = 0.49, aspect ratio 2, read as a 2D box (the
paper does not state the dimension).  The flow settles into steady
convection.  The table has two columns: the compared study's values (2.1,
26.3), which are what the validation is against and what the paper claims to
match within 3%, and the paper's own run (2.175, 26.98), itself 3.6% and 2.6%
above them.  The time means of Nu_bar (Eq. mean_Nu) and Re over the second
half of 150 time units must agree with the first column within 3% and with
the second within 5%.  Measured here (FP32, 128 x 64):
Nu_bar 2.093, Re 26.15 (0.4% and 0.6% below the reference values; 3.8% and
3.1% below the paper's own 2.175 and 26.98).  Grid-converged: FP64 at the
same grid and FP32 at 256 x 128 give 2.088-2.089 and 26.09-26.15.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_case1.json")


def test_table2_case1_nu_and_re():
    import paper_2411_10372_gb300 as cm
    g = json.load(open(GOLDEN))
    p = g["parameters"]
    s = cm.Solver(128, 64, p["Ra"], p["Pr"], p["gamma"], aspect=p["aspect"], precision="fp32", eps=p["eps"],
                  D=p["D"], t_top=1.0 - p["eps"] - p["D"], pert_amp=1e-2, diag_every=200, diag_capacity=1 << 14)
    try:
        hist = []
        while not hist or hist[-1][0] < 150.0:
            s.step(10000)
            hist += [(d["t"], d["Nu_bar"], d["Re"], d["status"]) for d in s.diagnostics()]
    finally:
        s.close()
    h = np.array(hist)
    assert np.all(h[:, 3] == 0)
    late = h[h[:, 0] > 0.5 * h[-1, 0]]
    nu, re = late[:, 1].mean(), late[:, 2].mean()
    tol = g["agreement_claimed_pct"] / 100.0
    # the table's two columns: the compared study's values (the validation
    # target the paper claims 3% agreement with) and the paper's own run
    dev = {"reference": (nu / g["reference_Nu"] - 1.0, re / g["reference_Re"] - 1.0),
           "paper": (nu / g["paper_Nu"] - 1.0, re / g["paper_Re"] - 1.0)}
    print("Table 2 case 1: Nu_bar %.4f Re %.3f; deviation from the reference column %s, from the paper's own %s"
          % (nu, re, dev["reference"], dev["paper"]))
    assert abs(dev["reference"][0]) <= tol and abs(dev["reference"][1]) <= tol, dev
    # the paper's own values sit 3.6% (Nu) and 2.6% (Re) above the reference
    # column, so a run within 1.3% of the reference is within 5% of them
    assert abs(dev["paper"][0]) <= 0.05 and abs(dev["paper"][1]) <= 0.05, dev
    # steady: the late samples do not drift
    assert late[:, 1].std() <= 1e-3 * nu and late[:, 2].std() <= 1e-3 * re
