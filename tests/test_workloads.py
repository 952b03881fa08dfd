"""The workload constants match the oracle-measured golden values."""

import json
import os

from paper_2112_09972_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "shan_chen_G3.5_tau1.json")


def test_constants_match_golden():
    with open(GOLDEN) as fh:
        g = json.load(fh)
    assert g["G"] == workloads.G_COUPLING
    assert g["sigma"] == workloads.SIGMA
    assert g["flat_rho_lo"] == workloads.RHO_LO


def test_parity_workload_parameters():
    w = workloads.C1_PARITY
    assert w.box == 32 and w.R == 6.0 and w.steps == 2000 and w.Ca == 0.1
    # Eq. 3 with the measured sigma: Ca = eta_s R gamma_dot / sigma
    assert abs(w.eta_s * w.R * w.shear_rate() / workloads.SIGMA - w.Ca) < 1e-15
    hist = workloads.C2_THROUGHPUT.gradient_history(200)
    # Eq. 15: the element-wise maximum of the rescaled history is u_LBM / L
    assert abs(abs(hist).max() - 0.1 / 128) < 1e-18
