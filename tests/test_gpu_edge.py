"""Empty and degenerate inputs of the GPU path: zero steps, a box without
droplet phase, and empty batches of the surrogate's network."""

import numpy as np
import pytest

from paper_2112_09972_gb300 import workloads
from paper_2112_09972_gb300.lbm import DropletLBM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev"])
def test_zero_steps_leave_the_state_unchanged(built, precision):
    g = DropletLBM((32, 16, 12), 3.0, (0.5 / 3, 0.5 / 3), 3.5, precision=precision, rho_hi=1.0,
                   rho_lo=workloads.RHO_LO)
    g.set_gradient(np.array([[0.0, 0.01, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), 0)
    g.step(3)
    f = g.populations()
    g.step(0)
    assert g.step_count() == 3
    assert np.array_equal(g.populations(), f)


def test_box_without_droplet_phase(built):
    """Pure solvent (rho_A = rho_lo, rho_B = 1 at rest everywhere): the droplet
    weight w = max(phi, 0) vanishes, so the moments are exactly zero, the
    second-moment tensor and D are undefined (NaN) and there is no component."""
    from oracle import lbm as olbm

    box = (32, 16, 12)
    _, w = olbm.lattice()
    ra = np.full(box[::-1], workloads.RHO_LO)
    rb = np.ones(box[::-1])
    f = np.stack([w[:, None, None, None] * ra[None], w[:, None, None, None] * rb[None]])
    g = DropletLBM(box, 3.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp32", rho_hi=1.0, rho_lo=workloads.RHO_LO)
    g.set_populations(f)
    assert np.all(g.moments() == 0.0)
    D, axes, lam, c = g.deformation()
    assert np.isnan(D) and np.all(np.isnan(lam)) and np.all(np.isnan(c))
    assert g.components()[0] == 0
    # the state stays droplet-free and finite under the ghost boundary at rest
    g.step(5)
    mass, _ = g.checksums()
    assert np.all(np.isfinite(mass)) and g.components()[0] == 0


def test_empty_batches_of_the_network(built):
    import torch

    from paper_2112_09972_gb300 import surrogate
    from paper_2112_09972_gb300.lbm import MLP

    net = MLP((576, 256, 6), max_batch=256, seed=1)
    x = torch.empty((0, 576), dtype=torch.float32, device="cuda")
    y = torch.empty((0, 6), dtype=torch.float32, device="cuda")
    D = torch.empty(0, dtype=torch.float64, device="cuda")
    net.forward(x, y)
    net.deformation(x, y, D)
    net.sync()
    net.close()
    sur = surrogate.Surrogate(max_batch=256)
    M, Dp = sur.predict(np.zeros((0, 576), dtype=np.float32))
    assert M.shape == (0, 6) and Dp.shape == (0,)
    sur.close()


def test_bounded_wait_gives_up_and_the_device_stays_usable(built):
    """Failure path of the device-side waits without a GPU fault: a warp waits
    on an mbarrier that nothing arrives on; the bounded wait gives up after
    its limit, the call reports LBM_ETIMEOUT, and the device then runs a
    normal step.  A barrier that does complete reports success."""
    import time

    from paper_2112_09972_gb300.lbm import selftest_wait

    t0 = time.perf_counter()
    assert selftest_wait(5_000_000) == -6  # LBM_ETIMEOUT after 5 ms
    assert time.perf_counter() - t0 < 5.0
    assert selftest_wait(5_000_000, arrive=True) == 0
    assert selftest_wait(10) == -1  # limit below 1 us: LBM_EINVAL
    g = DropletLBM((32, 16, 12), 3.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp32", rho_hi=1.0, rho_lo=workloads.RHO_LO)
    g.step(2)
    g.sync()
    assert np.isfinite(g.deformation()[0])
