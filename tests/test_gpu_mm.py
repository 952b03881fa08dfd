"""The GPU-batched Maffettone-Minale integrator (lbm_mm_integrate) against the
float64 model of oracle/mm.py (itself pinned to the steady simple-shear closed
form and the Taylor limit).

The same RK4 with the same step, the table read linearly in between rows on
both sides: float64 agrees to 1e-12 (rounding order only), float32 to 1e-5
in D (float32 rounding over a few thousand steps of a contracting flow).
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


def _reference(table, tau_d, chi, substeps, record_every):
    from oracle import mm

    T = table.shape[0]

    def grad(t):
        lo = min(int(np.floor(t)), T - 2)
        w = t - lo
        return (1.0 - w) * table[lo] + w * table[lo + 1]

    out = []
    for r in range(0, T, record_every):
        if r == 0:
            out.append(0.0)
            continue
        M, _, _ = mm.integrate(grad, float(r), tau_d, chi, h=1.0 / substeps)
        out.append(mm.deformation(M))
    return np.array(out)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_matches_float64_model(built, precision, tol):
    import torch

    from paper_2112_09972_gb300.lbm import mm_integrate

    T, n, tau_d, chi, sub, rec = 121, 3, 6.9, 1.0, 8, 40
    hist = np.stack([inputs.rescale_to_lattice(inputs.ou_gradient_history(T, 30.0, 1.0, 5, box_id=k), 0.1, 16)
                     for k in range(n)], axis=1)
    A = torch.from_numpy(np.ascontiguousarray(hist)).cuda()
    D = mm_integrate(A, tau_d, chi, substeps=sub, record_every=rec, precision=precision).cpu().numpy()
    for k in range(n):
        ref = _reference(hist[:, k], tau_d, chi, sub, rec)
        assert np.max(np.abs(D[:, k] - ref)) <= tol, (k, D[:, k], ref)


@pytest.mark.parametrize("Ca", [0.02, 0.2])
def test_steady_shear_closed_form(built, Ca):
    """Steady simple shear reaches the closed form of Maffettone & Minale,
    D = [sqrt(f1^2 + Ca^2) - sqrt(f1^2 + Ca^2 (1 - f2^2))] / (f2 Ca)."""
    import torch

    from paper_2112_09972_gb300.lbm import mm_integrate

    tau_d, chi = 5.0, 1.0
    gd = Ca / tau_d
    T = 400  # 80 droplet times
    A = torch.from_numpy(np.tile(inputs.simple_shear(gd), (T, 1, 1)).reshape(T, 1, 9).copy()).cuda()
    D = mm_integrate(A, tau_d, chi, substeps=4, record_every=T - 1).cpu().numpy()
    f1 = 40.0 * (chi + 1) / ((3 + 2 * chi) * (16 + 19 * chi))
    f2 = 5.0 / (3 + 2 * chi) + 3 * Ca ** 2 / (2 + 6 * Ca ** 2)
    ref = (np.sqrt(f1 ** 2 + Ca ** 2) - np.sqrt(f1 ** 2 + Ca ** 2 * (1 - f2 ** 2))) / (f2 * Ca)
    assert abs(D[-1, 0] / ref - 1.0) <= 1e-8


def test_invalid_arguments(built):
    import torch

    from paper_2112_09972_gb300.lbm import LBMError, mm_integrate

    A = torch.zeros((4, 2, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(LBMError):
        mm_integrate(A, -1.0, 1.0)
    with pytest.raises(LBMError):
        mm_integrate(A, 1.0, 1.0, substeps=0)
