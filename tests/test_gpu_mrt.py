"""The MRT collision on the GPU (the row kernel for float32 storage on
row-tiled shapes, the generic kernel otherwise) against the oracle's MRT
operator (oracle/lbm_oracle.cpp, pinned in tests/test_oracle_mrt.py).

Tolerances as for BGK (tests/test_gpu_parity.py): float64 differs by the
order of operations (1e-12 after 30 steps); float32 by its rounding (2e-5).
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads
from paper_2112_09972_gb300.lbm import DropletLBM

pytestmark = pytest.mark.gpu

RATES = (1.19, 1.4, 1.2, 1.4, 1.98)


@pytest.fixture(scope="session")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,tol,periodic,box", [
    ("fp64", 1e-12, False, (37, 29, 23)), ("fp64", 1e-12, True, (37, 29, 23)),
    ("fp32", 2e-5, False, (37, 29, 23)), ("fp32", 2e-5, True, (37, 29, 23)),
    ("fp32", 2e-5, False, (64, 24, 20)),    # the row kernel (64-wide rows, 3 clusters)
    ("fp32", 2e-5, False, (128, 16, 14))])  # the row kernel, 128-wide rows, one short z chunk
def test_mrt_matches_oracle(built, oracle_mod, precision, tol, periodic, box):
    tau = (0.9, 1.3)
    o = oracle_mod.OracleLBM(box, tau, 3.5, (workloads.RHO_LO, 1.0), periodic=periodic, mrt=RATES)
    g = DropletLBM(box, 5.0, ((tau[0] - 0.5) / 3, (tau[1] - 0.5) / 3), 3.5, precision=precision, periodic=periodic,
                   rho_hi=1.0, rho_lo=workloads.RHO_LO, mrt=RATES)
    hist = inputs.ou_gradient_history(30, 50.0, 300.0, seed=7)
    o.init_droplet(5.0, 1.0, 1.0, workloads.RHO_LO, hist[0])
    f0 = inputs.perturbed_populations(o.populations(), 1e-3, seed=3)
    o.set_populations(f0)
    g.set_populations(f0)
    g.set_gradient_table(np.arange(30), hist)
    for t in range(30):
        o.step(None if periodic else hist[t])
    g.step(30)
    assert rel_linf(g.populations(), o.populations()) <= tol


def test_mrt_default_rates_and_shape(built):
    """mrt=True takes the default free rates; with float32 storage on a
    row-tiled shape MRT runs on the row kernel (tile_y = 1 in the launch
    shape), with float64 storage on the generic kernel (tile_y > 1)."""
    w = workloads.C1_PARITY
    g64 = DropletLBM((32, 32, 32), w.R, w.visc, w.G, precision="fp64", rho_lo=w.rho_lo, mrt=True)
    assert g64.launch_shape()[0] > 1
    g64.close()
    g = DropletLBM((32, 32, 32), w.R, w.visc, w.G, precision="fp32", rho_lo=w.rho_lo, mrt=True)
    ty, _, _ = g.launch_shape()
    assert ty == 1
    g.set_gradient(inputs.simple_shear(w.shear_rate()), 0)
    g.step(200)
    D = g.deformation()[0]
    assert 0.01 < D < 0.3
