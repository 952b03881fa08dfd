"""Breakup detection (lbm_components): connected components of the droplet
phase phi > 0 against scipy.ndimage.label with 6-connectivity (exact: the
counts and the sorted component sizes are integers)."""

import numpy as np
import pytest

from paper_2112_09972_gb300 import workloads
from paper_2112_09972_gb300.lbm import DropletLBM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


def _rest_populations(ra, rb):
    """Rest equilibria w_i rho of the given densities, [2, 19, z, y, x]."""
    from oracle import lbm as olbm

    _, w = olbm.lattice()
    return np.stack([w[:, None, None, None] * ra[None], w[:, None, None, None] * rb[None]])


def _phase_fields(phi):
    lo, hi = workloads.RHO_LO, 1.0
    ra = lo + (hi - lo) * 0.5 * (1.0 + phi)
    rb = lo + (hi - lo) * 0.5 * (1.0 - phi)
    return ra, rb


def _scipy_components(mask, periodic=False):
    from scipy import ndimage

    lab, n = ndimage.label(mask, structure=ndimage.generate_binary_structure(3, 1))
    if periodic and n:
        # merge labels that touch across each periodic face (union-find on labels)
        parent = list(range(n + 1))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for ax in range(3):
            a = np.take(lab, 0, axis=ax)
            b = np.take(lab, -1, axis=ax)
            for u, v in zip(a[(a > 0) & (b > 0)], b[(a > 0) & (b > 0)]):
                ru, rv = find(int(u)), find(int(v))
                if ru != rv:
                    parent[max(ru, rv)] = min(ru, rv)
        roots = np.array([find(int(v)) for v in range(n + 1)])
        lab = roots[lab]
        lab[~mask] = 0
    ids, counts = np.unique(lab[lab > 0], return_counts=True)
    return len(ids), np.sort(counts)[::-1]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_blobs_match_scipy(built, precision, seed):
    from scipy import ndimage

    box = (32, 24, 20)
    rng = np.random.default_rng(seed)
    phi = ndimage.gaussian_filter(rng.normal(size=box[::-1]), 1.0)
    phi = np.tanh(phi / phi.std() * 2.0 - 0.8)  # 20 to 30 blobs
    ra, rb = _phase_fields(phi)
    f = _rest_populations(ra, rb)
    g = DropletLBM(box, 2.0, (0.5 / 3, 0.5 / 3), 3.5, precision=precision, rho_hi=1.0, rho_lo=workloads.RHO_LO)
    g.set_populations(f)
    fra, frb, _ = g.fields()
    mask = (fra - frb) / (fra + frb) > 0.0  # the phase of the state the library holds
    n_ref, sizes_ref = _scipy_components(mask)
    assert n_ref >= 10
    n, sizes = g.components(0.0, 1, max_sizes=len(sizes_ref) + 2)
    assert n == n_ref
    assert np.array_equal(sizes[:n], sizes_ref)
    assert np.all(sizes[n:] == 0)
    # the size filter
    n5, _ = g.components(0.0, 5, max_sizes=1)
    assert n5 == int(np.sum(sizes_ref >= 5))


def test_two_droplets_and_periodic_wrap(built):
    box = (40, 32, 32)
    z, y, x = np.meshgrid(*[np.arange(v) for v in box[::-1]], indexing="ij")

    def sphere(cx, cy, cz, r):
        return np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - r

    d = np.minimum(sphere(10, 16, 16, 6), sphere(30, 16, 16, 6))
    ra, rb = _phase_fields(-np.tanh(d))
    g = DropletLBM(box, 4.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp32", rho_hi=1.0, rho_lo=workloads.RHO_LO)
    g.set_populations(_rest_populations(ra, rb))
    n, sizes = g.components()
    assert n == 2 and abs(int(sizes[0]) - int(sizes[1])) <= 2
    # a blob cut by the x faces: two pieces in a walled box, one when periodic
    d = sphere(0, 16, 16, 7)
    d = np.minimum(d, sphere(40, 16, 16, 7))
    ra, rb = _phase_fields(-np.tanh(d))
    f = _rest_populations(ra, rb)
    walled = DropletLBM(box, 4.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp32", rho_hi=1.0, rho_lo=workloads.RHO_LO)
    walled.set_populations(f)
    per = DropletLBM(box, 4.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp32", periodic=True, rho_hi=1.0,
                     rho_lo=workloads.RHO_LO)
    per.set_populations(f)
    fra, frb, _ = per.fields()
    mask = (fra - frb) / (fra + frb) > 0.0
    assert walled.components()[0] == _scipy_components(mask)[0] == 2
    n_per, sizes_per = per.components()
    n_ref, sizes_ref = _scipy_components(mask, periodic=True)
    assert n_per == n_ref == 1 and sizes_per[0] == sizes_ref[0]


def test_droplet_stays_whole_in_gentle_shear(built):
    """The parity droplet under Ca = 0.1 shear stays one component."""
    w = workloads.C1_PARITY
    from paper_2112_09972_gb300 import inputs

    g = DropletLBM((w.box,) * 3, w.R, w.visc, w.G, precision="fp32", rho_hi=w.rho_hi, rho_lo=w.rho_lo)
    g.set_gradient(inputs.simple_shear(w.shear_rate()), 0)
    g.step(500)
    n, sizes = g.components(0.0, 10)
    assert n == 1 and sizes[0] > 500
