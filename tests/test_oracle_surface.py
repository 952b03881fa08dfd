"""Pins of the oracle's Eq. 17 surface-area deformation and of its mass
reinjection (oracle/observables.py).

* Eq. 17 on diffuse tanh-profile shapes of known geometry: the co-area
  surface area of a sphere and of prolate spheroids within 1.5 % of the
  closed forms (4 pi R^2; 2 pi b^2 (1 + a arcsin(e) / (b e))), the volume
  within 5 % (the diffuse interface adds a shell of order R^2 xi), D_LBM of
  the sphere 0, and D_LBM within 0.05 of the closed form and increasing
  with the aspect ratio;
* reinjection: the droplet component's total mass becomes the target, the
  populations outside phi > 0 and those of the other component are
  untouched, and those inside are scaled by one factor.
"""

import numpy as np
import pytest


def _shape(box, a, b, c, xi=1.0):
    """Densities of a diffuse ellipsoid: phi = tanh(d / xi), d the distance
    estimate (1 - r) min(a, b, c) with r the ellipsoidal radius."""
    z, y, x = np.meshgrid(*[np.arange(n) - 0.5 * (n - 1) for n in box[::-1]], indexing="ij")
    r = np.sqrt((x / a) ** 2 + (y / b) ** 2 + (z / c) ** 2)
    phi = np.tanh((1.0 - r) * min(a, b, c) / xi)
    lo = 0.0024
    return lo + (1 - lo) * 0.5 * (1 + phi), lo + (1 - lo) * 0.5 * (1 - phi)


def _spheroid(a, b):
    e = np.sqrt(1.0 - b * b / (a * a))
    area = 2 * np.pi * b * b * (1 + a * np.arcsin(e) / (b * e))
    vol = 4.0 / 3.0 * np.pi * a * b * b
    return area, vol, np.sqrt(1 - (36 * np.pi * vol * vol) ** (1 / 3) / area)


def test_sphere():
    from oracle.observables import surface_deformation

    D, area, vol = surface_deformation(*_shape((48, 48, 48), 10, 10, 10))
    assert abs(area / (4 * np.pi * 100) - 1) <= 0.015
    assert abs(vol / (4 / 3 * np.pi * 1000) - 1) <= 0.05
    assert D <= 0.02


@pytest.mark.parametrize("a,b,box", [(14, 9, (48, 48, 48)), (20, 8, (64, 48, 48))])
def test_prolate_spheroids(a, b, box):
    from oracle.observables import surface_deformation

    D, area, vol = surface_deformation(*_shape(box, a, b, b))
    A_ref, V_ref, D_ref = _spheroid(a, b)
    assert abs(area / A_ref - 1) <= 0.015
    assert abs(vol / V_ref - 1) <= 0.05
    assert abs(D - D_ref) <= 0.05


def test_deformation_grows_with_aspect_ratio():
    from oracle.observables import surface_deformation

    Ds = [surface_deformation(*_shape((64, 48, 48), a, b, b))[0] for a, b in [(11, 10), (14, 9), (17, 8.5), (20, 8)]]
    assert all(d2 > d1 for d1, d2 in zip(Ds, Ds[1:]))


def test_reinjection():
    from oracle.observables import phase_field, reinject_mass

    rng = np.random.default_rng(4)
    ra, rb = _shape((20, 18, 16), 6, 5, 5)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = np.stack([w[:, None, None, None] * ra[None], w[:, None, None, None] * rb[None]])
    f *= 1.0 + 0.01 * rng.standard_normal(f.shape)
    target = 1.05 * f[0].sum()
    g = reinject_mass(f, target)
    assert abs(g[0].sum() / target - 1) <= 1e-14
    inside = phase_field(f[0].sum(0), f[1].sum(0)) > 0
    assert np.array_equal(g[1], f[1])
    assert np.array_equal(g[0][:, ~inside], f[0][:, ~inside])
    ratio = g[0][:, inside] / f[0][:, inside]
    assert np.allclose(ratio, ratio.flat[0], rtol=1e-14, atol=0)
