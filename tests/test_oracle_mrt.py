"""Pins of the oracle's MRT collision (the multi-relaxation-time operator that
Sec. 2 names; d'Humieres et al. 2002 moment basis).

* The basis: rows mutually orthogonal, with the squared norms published for
  D3Q19 (19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8,
  8); the first rows are 1, c_x, c_y, c_z (density and momentum).
* With every rate equal to 1/tau the operator is BGK, state for state.
* Periodic mode with the Shan-Chen force, tau_A != tau_B and the published
  free rates: mass of each component and total momentum conserved.
* A shear wave decays at nu k^2 with nu = (tau - 1/2)/3 set by the stress
  rates alone: the free rates do not change it (Eq. 10).
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads

NORMS = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]


def test_basis_orthogonal_with_published_norms(oracle_mod):
    from oracle import lbm as olbm

    M = olbm.moment_basis()
    c, _ = olbm.lattice()
    G = M @ M.T
    assert np.array_equal(np.diag(G), np.array(NORMS, dtype=np.float64))
    assert np.max(np.abs(G - np.diag(np.diag(G)))) == 0.0
    assert np.array_equal(M[0], np.ones(19))
    for row, a in ((3, 0), (5, 1), (7, 2)):
        assert np.array_equal(M[row], c[:, a].astype(np.float64))


def _perturbed(oracle_mod, box, periodic, seed):
    o = oracle_mod.OracleLBM(box, (0.9, 1.3), 3.5, (workloads.RHO_LO, 1.0), periodic=periodic)
    A = inputs.simple_shear(0.01)
    o.init_droplet(3.0, 1.0, 1.0, workloads.RHO_LO, A)
    return inputs.perturbed_populations(o.populations(), 1e-3, seed=seed), A


def test_equal_rates_is_bgk(oracle_mod):
    box = (12, 10, 11)
    f0, A = _perturbed(oracle_mod, box, False, 3)
    # the operator takes one free-rate set for both components; use equal taus
    bgk = oracle_mod.OracleLBM(box, (1.1, 1.1), 3.5, (workloads.RHO_LO, 1.0))
    mrt = oracle_mod.OracleLBM(box, (1.1, 1.1), 3.5, (workloads.RHO_LO, 1.0), mrt=(1 / 1.1,) * 5)
    bgk.set_populations(f0)
    mrt.set_populations(f0)
    for _ in range(5):
        bgk.step(A)
        mrt.step(A)
    assert np.max(np.abs(mrt.populations() - bgk.populations())) <= 1e-14


def test_periodic_conservation(oracle_mod):
    from oracle import lbm as olbm

    box = (12, 10, 11)
    f0, _ = _perturbed(oracle_mod, box, True, 5)
    o = oracle_mod.OracleLBM(box, (0.9, 1.3), 3.5, (workloads.RHO_LO, 1.0), periodic=True, mrt=olbm.MRT_RATES)
    o.set_populations(f0)
    m0, p0 = o.checksums()
    o.run(40)
    m1, p1 = o.checksums()
    assert np.all(np.abs(m1 - m0) <= 1e-13 * m0)
    assert np.all(np.abs(p1 - p0) <= 1e-13 * m0.sum())


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_shear_wave_set_by_stress_rates(oracle_mod, tau):
    from oracle import lbm as olbm

    L, U = 128, 1e-3
    rates = {}
    for name, mrt in (("bgk", None), ("dh", olbm.MRT_RATES), ("other", (1.6, 1.1, 1.5, 1.7, 1.2))):
        o = oracle_mod.OracleLBM((1, L, 1), (tau, tau), 0.0, (0.5, 0.5), periodic=True, mrt=mrt)
        y = np.arange(L)
        f = np.zeros(o.shape)
        for n in range(L):
            u = np.array([U * np.sin(2 * np.pi * y[n] / L), 0.0, 0.0])
            for i in range(19):
                g = oracle_mod.equilibrium(i, 0.5, u)
                f[0, i, 0, n, 0] = g
                f[1, i, 0, n, 0] = g
        o.set_populations(f)
        k = 2 * np.pi / L
        s, c = np.sin(k * y), np.cos(k * y)

        def amp():
            ux = o.fields()[2][0, :, 0, 0]
            return np.hypot(ux @ s, ux @ c) * 2 / L

        o.run(50)
        a1 = amp()
        o.run(400)
        rates[name] = -np.log(amp() / a1) / 400
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / L
    for name in ("dh", "other"):
        assert abs(rates[name] / (nu * k * k) - 1.0) < 8e-3, name
        assert abs(rates[name] / rates["bgk"] - 1.0) < 2e-3, name
