"""Pins of the FP64 oracle that hold exactly (to round-off).

Each test checks the oracle against a fact fixed by mathematics or by the
paper's equations, not by re-typing the oracle's own formula:

* D3Q19 moment identities (weights of Eq. 7/8; isotropy to fourth order);
* moments of the equilibrium of Eq. 8;
* the rest state with ghost nodes (Sec. 2, Eq. 8) is a fixed point;
* a simple shear u = A x (A^2 = 0) of a uniform mixture is a fixed point of
  stream + ghost boundary + collision at tau = 1 (shown analytically in the
  docstring of ``test_simple_shear_preserved_exactly``);
* periodic mode conserves each component's mass and the total momentum
  (Eq. 7's force sums to zero over a periodic box, and the tau-weighted common
  velocity makes the collision exchange no momentum beyond F);
* with ghost nodes the change of mass equals the inflow from ghosts minus the
  post-collision outflow, exactly.
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs


def test_lattice_identities(oracle_mod):
    c, w = oracle_mod.lattice()
    assert c.shape == (19, 3)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    # speeds: 1 rest, 6 of |c|^2=1, 12 of |c|^2=2; every vector has its opposite
    c2 = (c ** 2).sum(1)
    assert sorted(c2.tolist()) == [0] + [1] * 6 + [2] * 12
    for i in range(19):
        assert any((c[j] == -c[i]).all() for j in range(19))
    # first, second, third and fourth moments of the weights
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)
    # weights by speed: 1/3, 1/18, 1/36
    assert np.allclose(w[c2 == 0], 1 / 3) and np.allclose(w[c2 == 1], 1 / 18) and np.allclose(w[c2 == 2], 1 / 36)


def test_equilibrium_moments(oracle_mod):
    c, _ = oracle_mod.lattice()
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = rng.uniform(0.01, 2.0)
        u = rng.uniform(-0.2, 0.2, size=3)
        geq = np.array([oracle_mod.equilibrium(i, rho, u) for i in range(19)])
        assert np.isclose(geq.sum(), rho, rtol=1e-14)
        assert np.allclose(geq @ c, rho * u, rtol=0, atol=1e-15)
        # second moment: rho (c_s^2 delta + u u), exact for the D3Q19 second-order equilibrium
        P = np.einsum("i,ia,ib->ab", geq, c, c)
        assert np.allclose(P, rho * (np.eye(3) / 3 + np.outer(u, u)), rtol=0, atol=1e-15)


def _uniform_mixture(oracle_mod, box, rho_a, rho_b, A=None):
    o_tmp = oracle_mod.OracleLBM(box, (1.0, 1.0), 0.0, (rho_a, rho_b))
    # a droplet of radius 0 with rho_hi == rho_lo is a uniform state
    o_tmp.init_droplet(0.0, 1.0, rho_a, rho_a, A)
    fa = o_tmp.populations()[0]
    o_tmp.init_droplet(0.0, 1.0, rho_b, rho_b, A)
    fb = o_tmp.populations()[1]
    return np.stack([fa, fb])


def test_rest_state_is_fixed_point(oracle_mod):
    box = (6, 7, 5)
    rho_a, rho_b = 0.034, 1.0
    f0 = _uniform_mixture(oracle_mod, box, rho_a, rho_b)
    o = oracle_mod.OracleLBM(box, (0.8, 1.7), 3.5, (rho_a, rho_b))
    o.set_populations(f0)
    for _ in range(10):
        o.step(np.zeros(9))
    assert np.max(np.abs(o.populations() - f0)) <= 1e-16


def test_simple_shear_preserved_exactly(oracle_mod):
    """u = A x with A = g e_x e_y^T is a fixed point at tau = 1.

    At tau = 1 the post-collision populations are equilibria, exactly like the
    ghost populations, so after streaming every node holds
    g^eq_i(rho, A (x - c_i)).  Using the D3Q19 moments up to fourth order, the
    density of that set is rho (1 + tr(A A)/2) and its momentum rho (I - A) A x;
    for A^2 = 0 these are rho and rho A x, the force of a uniform mixture is
    zero, and the collision restores g^eq(rho, A x).  Any error in the ghost
    geometry, the streaming direction or the equilibrium breaks this.
    """
    box = (8, 9, 7)
    A = inputs.simple_shear(0.02)
    rho_a, rho_b = 0.05, 0.97
    f0 = _uniform_mixture(oracle_mod, box, rho_a, rho_b, A)
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (rho_a, rho_b))
    o.set_populations(f0)
    for _ in range(30):
        o.step(A)
    assert np.max(np.abs(o.populations() - f0)) <= 1e-15
    ra, rb, u = o.fields()
    from oracle.observables import positions

    assert np.max(np.abs(u - positions(box) @ A.reshape(3, 3).T)) <= 1e-14


def test_planar_extension_changes_density_by_trace_of_A_squared(oracle_mod):
    """For A^2 != 0 the streamed density is rho (1 + tr(A A)/2) at tau = 1 (one step)."""
    box = (6, 6, 6)
    e = 0.01
    A = np.diag([e, -e, 0.0]).reshape(9)
    rho = 0.9
    f0 = _uniform_mixture(oracle_mod, box, rho, rho, A)
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 0.0, (rho, rho))
    o.set_populations(f0)
    o.step(A)
    ra, rb, _ = o.fields()
    expect = rho * (1.0 + 0.5 * np.trace(A.reshape(3, 3) @ A.reshape(3, 3)))
    assert np.allclose(ra, expect, rtol=1e-14) and np.allclose(rb, expect, rtol=1e-14)


def test_periodic_mode_conserves_mass_and_momentum(oracle_mod):
    box = (12, 10, 11)
    from oracle.observables import coexistence_rho_lo

    lo = coexistence_rho_lo(3.5)
    o = oracle_mod.OracleLBM(box, (0.9, 1.3), 3.5, (lo, 1.0), periodic=True)
    o.init_droplet(3.5, 1.0, 1.0, lo, inputs.simple_shear(0.01))
    o.set_populations(inputs.perturbed_populations(o.populations(), 1e-3, seed=11))
    m0, p0 = o.checksums()
    for _ in range(40):
        o.step()
    m1, p1 = o.checksums()
    assert np.all(np.abs(m1 - m0) <= 1e-13 * m0)
    assert np.all(np.abs(p1 - p0) <= 1e-13 * m0.sum())


def test_ghost_boundary_mass_bookkeeping(oracle_mod):
    box = (10, 9, 8)
    from oracle.observables import coexistence_rho_lo

    lo = coexistence_rho_lo(3.5)
    A = inputs.ou_gradient_history(5, 100.0, 40.0, seed=5)
    o = oracle_mod.OracleLBM(box, (1.0, 1.2), 3.5, (lo, 1.0))
    o.init_droplet(3.0, 1.0, 1.0, lo, A[0])
    for t in range(5):
        m0, _ = o.checksums()
        fin, fout = o.step(A[t], fluxes=True)
        m1, _ = o.checksums()
        assert np.all(np.abs((m1 - m0) - (fin - fout)) <= 1e-13 * m0)
        assert np.all(fin > 0) and np.all(fout > 0)
