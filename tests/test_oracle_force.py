"""Pins of the oracle's Shan-Chen force (Sec. 2, Eq. 7) and of the velocity-shift
forcing that carries it into the collision, against closed forms.

One step, exactly.  Component A uniform (rho_A0), component B a small
sinusoid rho_B = rho0 + eps sin(k s) along a lattice direction, both at rest
equilibrium (g_i = w_i rho), periodic box.  One step of the method is then a
closed form that follows from the D3Q19 weights alone:

* streaming moves B's populations by -c_i, so B's density keeps its shape
  with amplitude eps' = eps * a(k) and picks up the momentum
  j_B = -2 eps b(k) cos(k s) along the wave, where a and b are the weighted
  sums of cos(k m) and sin(k m) over the lattice directions by their
  projection m = c_i . e onto the wave (e the unit steps of the wave);
* Eq. 7 on the streamed densities: F^A = -G rho_A0 sum_i w_i rho_B'(x + c_i) c_i
  = -G rho_A0 * 2 eps' b(k) cos(k s) along the wave, F^B = 0 (A is uniform);
* the common velocity u' = (j_B / tau_B) / (rho_A0 / tau_A + rho_B' / tau_B),
  the shifted equilibrium velocities u_s = u' + tau_s F^s / rho_s, and BGK
  relaxation (Eqs. 9, 10) give the stored momenta
  j*_A = rho_A0 u' / tau_A + F^A,   j*_B = j_B (1 - 1/tau_B) + rho_B' u' / tau_B.
Any error in the force's magnitude, sign, weights, neighbour offsets or
velocity shift moves j*_A by a fraction of F^A, far above FP64 rounding.

Flat-interface coexistence.  In the steady state of a flat interface each
component carries no mass flux.  Streaming moves the post-collision momentum
minus half the gradient of the momentum flux, (c_s^2 / 2) grad rho_s, and
one step of the velocity-shift forcing relaxes the momentum towards
rho_s u' + tau_s F^s.  To first order in the gradients the zero-flux
condition of component A is
    (tau - 1/2) grad ln rho_A + (1/2) grad ln(rho_A + rho_B) = -tau G grad rho_B,
whose integral across the interface between the symmetric bulk phases
(h, l) and (l, h) is
    ln(h / l) = G tau / (tau - 1/2) * (h - l).
The continuum balance c_s^2 grad rho_A = -G c_s^2 rho_A grad rho_B, i.e.
ln(h/l) = G (h - l), is its limit tau -> infinity; at tau = 1 the discrete
model's effective coupling is 2 G.  Near the critical point the interface is
wide and the higher-order gradient terms vanish, so the relation holds to a
fraction of a percent there.
"""

import numpy as np
import pytest
from scipy.optimize import brentq


def _rest_populations(oracle_mod, shape, rho_a, rho_b):
    """Rest equilibria g_i = w_i rho (Eq. 8 at u = 0) of two density fields."""
    f = np.zeros(shape)
    for i in range(19):
        w = oracle_mod.equilibrium(i, 1.0, (0.0, 0.0, 0.0))
        f[0, i] = w * rho_a
        f[1, i] = w * rho_b
    return f


def _momentum(oracle_mod, f):
    """sum_i f_i c_i per component, shaped [2, z, y, x, 3]."""
    c = oracle_mod.lattice()[0]
    return np.einsum("sizyx,ia->szyxa", f, c.astype(float))


def _one_step(oracle_mod, box, tau, G, rho_a0, rho_b):
    o = oracle_mod.OracleLBM(box, tau, G, (0.1, 0.1), periodic=True)
    shape = o.shape
    f0 = _rest_populations(oracle_mod, shape, np.full(shape[2:], rho_a0), rho_b)
    o.set_populations(f0)
    o.step()
    f1 = o.populations()
    return f1.sum(axis=1), _momentum(oracle_mod, f1)


# Weighted sums of the D3Q19 weights by m = c_i . e for a wave along e:
#   axis wave e = (1, 0, 0): weight of m = 0 is 2/3, of m = +-1 is 1/6 each;
#   diagonal wave e = (1, 1, 0): m = 0: 1/2, m = +-1: 2/9, m = +-2: 1/36.
# a(k) = sum_m W_m cos(k m) (streamed density amplitude per unit amplitude);
# b(k) = sum over directions with c_i . x = +1 of w_i sin(k m_i), so that
#   sum_i w_i c_ix sin(phi + k m_i) = 2 b(k) cos(phi).
def _axis_ab(k):
    return 2.0 / 3.0 + 2.0 / 6.0 * np.cos(k), np.sin(k) / 6.0


def _diag_ab(k):
    return 0.5 + 4.0 / 9.0 * np.cos(k) + 1.0 / 18.0 * np.cos(2 * k), np.sin(k) / 9.0 + np.sin(2 * k) / 36.0


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.3)])
def test_one_step_axis_wave_matches_closed_form(oracle_mod, axis, tau):
    L, m, eps, rho0, rho_a0, G = 24, 2, 0.02, 0.6, 0.45, 1.7
    k = 2 * np.pi * m / L
    box = [1, 1, 1]
    box[axis] = L
    s = np.arange(L, dtype=float).reshape([L if a == axis else 1 for a in (2, 1, 0)])
    rho_b = np.broadcast_to(rho0 + eps * np.sin(k * s), (box[2], box[1], box[0]))
    rho, j = _one_step(oracle_mod, tuple(box), tau, G, rho_a0, rho_b)
    a, b = _axis_ab(k)
    eps1 = eps * a
    rho_b1 = rho0 + eps1 * np.sin(k * s)
    jB = -2 * eps * b * np.cos(k * s)
    FA = -G * rho_a0 * 2 * eps1 * b * np.cos(k * s)
    tA, tB = tau
    up = (jB / tB) / (rho_a0 / tA + rho_b1 / tB)
    jA_star = rho_a0 * up / tA + FA
    jB_star = jB * (1 - 1 / tB) + rho_b1 * up / tB
    scale = np.max(np.abs(FA))
    assert scale > 1e-4
    # densities: BGK keeps each component's mass per node
    assert np.max(np.abs(rho[0] - rho_a0)) < 1e-15
    assert np.max(np.abs(rho[1] - rho_b1)) < 1e-15
    # momenta along the wave, and none across it
    assert np.max(np.abs(j[0][..., axis] - jA_star)) < 1e-12 * scale
    assert np.max(np.abs(j[1][..., axis] - jB_star)) < 1e-12 * scale
    others = [q for q in range(3) if q != axis]
    assert np.max(np.abs(j[:, ..., others])) < 1e-15


def test_one_step_diagonal_wave_matches_closed_form(oracle_mod):
    """A wave along x + y exercises the face-diagonal directions' weights."""
    L, m, eps, rho0, rho_a0, G, tau = 18, 1, 0.03, 0.5, 0.55, 2.1, (1.0, 1.0)
    k = 2 * np.pi * m / L
    y, x = np.meshgrid(np.arange(L, dtype=float), np.arange(L, dtype=float), indexing="ij")
    phi = (k * (x + y))[None]
    rho_b = rho0 + eps * np.sin(phi)
    rho, j = _one_step(oracle_mod, (L, L, 1), tau, G, rho_a0, rho_b)
    a, b = _diag_ab(k)
    eps1 = eps * a
    rho_b1 = rho0 + eps1 * np.sin(phi)
    jB = -2 * eps * b * np.cos(phi)
    FA = -G * rho_a0 * 2 * eps1 * b * np.cos(phi)
    up = jB / (rho_a0 + rho_b1)
    jA_star = rho_a0 * up + FA
    scale = np.max(np.abs(FA))
    assert np.max(np.abs(rho[1] - rho_b1)) < 1e-15
    for q in (0, 1):  # x and y components are equal for a wave along x + y
        assert np.max(np.abs(j[0][..., q] - jA_star)) < 1e-12 * scale
        assert np.max(np.abs(j[1][..., q] - rho_b1 * up)) < 1e-12 * scale
    assert np.max(np.abs(j[..., 2])) < 1e-15


def _first_order_lo(G, tau, h=1.0):
    Ge = G * tau / (tau - 0.5)
    return brentq(lambda l: np.log(h / l) - Ge * (h - l), 1e-12, 1.0 / Ge)


@pytest.mark.parametrize("G,tau,steps,tol", [(1.1, 1.0, 30000, 2e-3), (0.85, 0.8, 30000, 1.5e-2),
                                             (1.2, 2.0, 30000, 1.5e-2)])
def test_flat_coexistence_near_critical(oracle_mod, G, tau, steps, tol):
    """A relaxed flat slab's bulk densities satisfy ln(h/l) = G tau/(tau - 1/2) (h - l)."""
    L = 128
    lo0 = _first_order_lo(G, tau)
    o = oracle_mod.OracleLBM((L, 1, 1), (tau, tau), G, (lo0, 1.0), periodic=True)
    o.init_droplet(L / 4, 6.0, 1.0, lo0)
    o.run(steps)
    ra, rb, _ = o.fields()
    h, l = ra.max(), ra.min()
    # the two bulk phases are mirror images (A <-> B symmetry of the model)
    assert abs(rb.max() - h) < 1e-9 and abs(rb.min() - l) < 1e-9
    Ge = G * tau / (tau - 0.5)
    assert abs(np.log(h / l) / (Ge * (h - l)) - 1) < tol
    # the continuum relation (tau -> infinity) is far off at these tau
    assert abs(np.log(h / l) / (G * (h - l)) - 1) > 0.3
