"""Pins of the oracle's reduced models and observables.

* Maffettone-Minale (Sec. 2, Eqs. 1, 2, 5): its steady state in simple shear
  has the closed form of Maffettone & Minale (1998),
  D = [sqrt(f1^2 + Ca^2) - sqrt(f1^2 + Ca^2 (1 - f2^2))] / (f2 Ca),
  whose small-Ca limit is Taylor's law D = (19 chi + 16)/(16 chi + 16) Ca; the
  model conserves det M (droplet volume) for any traceless gradient.
* D from the inertia tensor (Eq. 4): a voxelised ellipsoid with semi-axes
  a > b > c has principal second moments ~ a_k^2/5, so D ~ (a - c)/(a + c);
  the moments agree with a brute-force numpy sum over the voxels.
* The synthetic gradient generator: traceless, <S:S> = <W:W> = 1/(2 tau_eta^2),
  lag-1 autocorrelation exp(-1/T).
"""

import numpy as np
import pytest

from oracle import mm
from oracle.observables import deformation_from_moments, conformation_tensor
from paper_2112_09972_gb300 import inputs


def _steady_shear_closed_form(chi, Ca):
    f1, f2 = mm.f1(chi), mm.f2(chi, Ca)
    return (np.sqrt(f1 ** 2 + Ca ** 2) - np.sqrt(f1 ** 2 + Ca ** 2 * (1 - f2 ** 2))) / (f2 * Ca)


@pytest.mark.parametrize("chi,Ca", [(1.0, 0.1), (1.0, 0.3), (0.5, 0.2), (3.0, 0.2)])
def test_mm_steady_shear_closed_form(chi, Ca):
    tau_d = 10.0
    G = np.zeros((3, 3))
    G[0, 1] = Ca / tau_d
    M, _, _ = mm.integrate(lambda t: G, 150 * tau_d, tau_d, chi, h=tau_d / 40)
    assert abs(mm.deformation(M) / _steady_shear_closed_form(chi, Ca) - 1) < 1e-8


@pytest.mark.parametrize("chi", [0.2, 1.0, 4.0])
def test_mm_taylor_limit(chi):
    Ca, tau_d = 0.005, 10.0
    G = np.zeros((3, 3))
    G[0, 1] = Ca / tau_d
    M, _, _ = mm.integrate(lambda t: G, 200 * tau_d, tau_d, chi, h=tau_d / 40)
    taylor = (19 * chi + 16) / (16 * chi + 16) * Ca
    assert abs(mm.deformation(M) / taylor - 1) < 2e-3


def test_mm_conserves_volume_and_sphere():
    hist = inputs.ou_gradient_history(2000, 200.0, 60.0, seed=3)
    ts = np.arange(len(hist), dtype=float)
    grad = lambda t: np.array([np.interp(t, ts, hist[:, j]) for j in range(9)]).reshape(3, 3)
    M, _, D = mm.integrate(grad, 1999.0, 15.0, 1.0, record_every=100)
    assert abs(np.linalg.det(M) - 1) < 1e-8
    assert D.max() > 0.01
    M0, _, _ = mm.integrate(lambda t: np.zeros((3, 3)), 100.0, 15.0, 1.0)
    assert np.allclose(M0, np.eye(3), atol=1e-14)


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_deformation_of_voxelised_ellipsoid(oracle_mod):
    L = 40
    a = np.array([12.0, 8.0, 6.0])
    Q = _rotation(9)
    box = (L, L, L)
    from oracle.observables import positions

    X = positions(box)
    body = X @ Q  # coordinates in the ellipsoid frame
    inside = np.sum((body / a) ** 2, axis=-1) <= 1.0
    hi, lo = 1.0, 0.05
    rho_a = np.where(inside, hi, lo)
    rho_b = np.where(inside, lo, hi)
    _, w = oracle_mod.lattice()
    f = np.stack([w[:, None, None, None] * rho_a[None], w[:, None, None, None] * rho_b[None]])
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 0.0, (lo, hi))
    o.set_populations(f)
    m = o.moments()
    # brute force over voxels: uniform weight phi_in inside, 0 outside
    phi_in = (hi - lo) / (hi + lo)
    P = X[inside]
    brute = np.array([inside.sum() * phi_in, *(phi_in * P.sum(0)),
                      *(phi_in * np.array([np.sum(P[:, i] * P[:, j]) for i, j in
                                           [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]]))])
    assert np.allclose(m, brute, rtol=1e-12, atol=1e-9)
    D, axes, lam, c = deformation_from_moments(m)
    assert np.allclose(np.sqrt(5 * lam), a, rtol=0.02)
    assert abs(D - (a[0] - a[2]) / (a[0] + a[2])) < 0.01
    for k in range(3):
        assert abs(abs(axes[:, k] @ Q[:, k]) - 1) < 1e-3
    M = conformation_tensor(m)
    assert abs(np.linalg.det(M) - 1) < 1e-12


def test_ou_gradient_statistics():
    T, tau_eta, n = 20.0, 3.0, 200000
    A = inputs.ou_gradient_history(n, T, tau_eta, seed=1).reshape(n, 3, 3)
    assert np.max(np.abs(np.trace(A, axis1=1, axis2=2))) < 1e-15
    S = 0.5 * (A + A.transpose(0, 2, 1))
    W = 0.5 * (A - A.transpose(0, 2, 1))
    ss = np.mean(np.sum(S * S, axis=(1, 2)))
    ww = np.mean(np.sum(W * W, axis=(1, 2)))
    target = 1.0 / (2 * tau_eta ** 2)
    assert abs(ss / target - 1) < 0.05 and abs(ww / target - 1) < 0.05
    a = A[:, 0, 1]
    rho1 = np.corrcoef(a[:-1], a[1:])[0, 1]
    assert abs(rho1 - np.exp(-1 / T)) < 5e-3
    # determinism: same seed and box id give the same history, another box id does not
    B = inputs.ou_gradient_history(50, T, tau_eta, seed=1)
    assert np.array_equal(B, inputs.ou_gradient_history(50, T, tau_eta, seed=1))
    assert not np.array_equal(B, inputs.ou_gradient_history(50, T, tau_eta, seed=1, box_id=1))
