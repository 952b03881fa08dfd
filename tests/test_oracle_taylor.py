"""The oracle's droplet in steady simple shear at small capillary number
(Sec. 2, Eqs. 1, 3, 4, 5; Sec. 5): Taylor's small-deformation regime.

Taylor's law D = (19 lambda + 16) / (16 lambda + 16) Ca (lambda = 1 here, so
35/32 Ca, with Ca = eta gamma_dot R / sigma of Eq. 3) describes three things
that a correct model reproduces at small Ca:

* the response is linear: doubling Ca doubles D;
* the major axis lies in the shear plane at 45 degrees to the flow, along
  the stretching direction of u_x = gamma_dot y, and the middle axis along
  the vorticity (z);
* the prefactor D / Ca.

The first two are held tightly here.  The prefactor of this model at tau = 1
lies above Taylor's by a factor that does not tend to 1 with resolution
(about 1.3-1.4 for R = 5..16, recorded with the measurements in the design
notes), so it is held to that band.  Measured on this case: the correct
model gives D / D_Taylor = 1.377 and 1.375 at 46.3 and 46.7 degrees; a
viscosity twice the one Ca assumes gives 1.59 and 1.72 at 43.7 and 42.6
degrees, and the transposed gradient (u_y = gamma_dot x) 43.7 and 43.3
degrees; a ghost flow that is not imposed leaves D near 0.  The force's
magnitude is pinned separately (test_oracle_force.py).

L = 40, R = 5: after 300 steps of the imposed flow (the droplet's relaxation
time eta R / sigma is a few steps; the flow is set in the initial state) D
has settled to within 1 %.
"""

import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "shan_chen_G3.5_tau1.json")


def _steady_shear(oracle_mod, L, R, Ca, steps, sigma, rho_lo):
    from oracle.observables import deformation_from_moments

    eta = 1.0 / 6.0  # rho nu with nu = (tau - 1/2) / 3 at tau = 1
    gamma_dot = Ca * sigma / (eta * R)
    A = np.zeros(9)
    A[1] = gamma_dot  # u_x = gamma_dot y
    o = oracle_mod.OracleLBM((L, L, L), (1.0, 1.0), 3.5, (rho_lo, 1.0))
    o.init_droplet(R, 1.0, 1.0, rho_lo, A)
    o.run(steps, [0.0], [A])
    D, axes, lam, _ = deformation_from_moments(o.moments())
    return D, axes


def test_small_ca_shear_is_in_taylors_regime(oracle_mod):
    with open(GOLDEN) as fh:
        g = json.load(fh)
    sigma, rho_lo = g["sigma"], g["flat_rho_lo"]
    L, R, steps = 40, 5.0, 300
    res = {Ca: _steady_shear(oracle_mod, L, R, Ca, steps, sigma, rho_lo) for Ca in (0.02, 0.04)}
    D1, D2 = res[0.02][0], res[0.04][0]
    # linear response
    assert 1.9 <= D2 / D1 <= 2.1, (D1, D2)
    for Ca, (D, axes) in res.items():
        # the prefactor: this model's band above Taylor's 35/32 at tau = 1
        assert 1.2 <= D / (35.0 / 32.0 * Ca) <= 1.5, (Ca, D)
        major, middle = axes[:, 0], axes[:, 1]
        # the major axis in the shear plane, along the stretching direction
        assert abs(major[2]) < 1e-3
        angle = np.degrees(np.arctan2(major[1], major[0]))
        assert 45.0 <= angle <= 49.0, (Ca, angle)
        # the middle axis along the vorticity
        assert abs(middle[2]) > 0.999, (Ca, middle)
