"""Observables of the FP64 oracle (test infrastructure only).

Each function restates one definition of the paper, or of the reading of it
that this repository adopts where the paper is silent:

* ``deformation_from_moments`` -- D = (L - W)/(L + W) (Sec. 2, Eq. 4) with the
  ellipsoid axes taken from the droplet's second-moment (inertia) tensor; a
  uniform ellipsoid with semi-axes a_k has principal second moments a_k^2/5,
  so the axes are proportional to sqrt(lambda_k).  The symmetric eigenproblem
  is solved by ``numpy.linalg.eigh`` (a library primitive).
* ``velocity_error_E0`` -- the global single-phase error E^(0)(t) (Sec. 4,
  Eq. 16).
* ``bulk_pressure`` -- p = c_s^2 (rho_A + rho_B) + G c_s^2 rho_A rho_B, the
  bulk equation of state of the Shan-Chen mixture of Eq. 7 with psi = rho.
* ``coexistence_rho_lo`` -- the minority density of a flat interface:
  ln(h/l) = G (h - l), the balance c_s^2 grad rho_A = -G c_s^2 rho_A grad rho_B
  that Eq. 7 gives in the continuum limit.
* ``surface_deformation`` -- D_LBM = sqrt(1 - Omega_0 / Omega) (Sec. 5,
  Eq. 17), with the surface area Omega of the diffuse interface read as the
  mean area of the level sets of phi between its extremes (the co-area
  formula: Omega = sum |grad phi| / (phi_max - phi_min), central differences
  at interior nodes) and Omega_0 = (36 pi V^2)^(1/3) the area of the sphere of
  the droplet's volume V = sum (phi - phi_min) / (phi_max - phi_min).
* ``reinject_mass`` -- the reading adopted for the mass reinjection that Sec. 2
  cites: the droplet component's populations at nodes with phi > 0 are
  multiplied by one factor, so that its total mass becomes the target.
"""

import numpy as np
from scipy.optimize import brentq

CS2 = 1.0 / 3.0


def inertia_tensor(m):
    """Centre of mass and central second-moment tensor from the 10 moments.

    ``m = {sum w, sum w x, sum w y, sum w z, sum w xx, sum w xy, sum w xz,
    sum w yy, sum w yz, sum w zz}``.
    """
    m = np.asarray(m, dtype=np.float64)
    mass = m[0]
    c = m[1:4] / mass
    S = np.array([[m[4], m[5], m[6]], [m[5], m[7], m[8]], [m[6], m[8], m[9]]]) / mass
    return c, S - np.outer(c, c)


def deformation_from_moments(m):
    """(D, axes[3,3] columns = principal axes, eigenvalues descending, centre).

    Each axis is sign-normalised so that its largest-magnitude component is
    positive.  D = (sqrt(l1) - sqrt(l3)) / (sqrt(l1) + sqrt(l3)).
    """
    c, I = inertia_tensor(m)
    lam, vec = np.linalg.eigh(I)
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    vec = vec[:, order]
    for k in range(3):
        j = np.argmax(np.abs(vec[:, k]))
        if vec[j, k] < 0:
            vec[:, k] = -vec[:, k]
    a1 = np.sqrt(max(lam[0], 0.0))
    a3 = np.sqrt(max(lam[2], 0.0))
    D = (a1 - a3) / (a1 + a3)
    return D, vec, lam, c


def conformation_tensor(m):
    """M = I / det(I)^(1/3): the unit-determinant shape tensor (delta for a sphere)."""
    _, I = inertia_tensor(m)
    return I / np.cbrt(np.linalg.det(I))


def bulk_pressure(rho_a, rho_b, G):
    return CS2 * (rho_a + rho_b) + G * CS2 * rho_a * rho_b


def coexistence_rho_lo(G, rho_hi=1.0):
    """Minority density l of the flat interface: ln(h/l) = G (h - l), l < 1/G."""
    h = float(rho_hi)
    if G * h <= 1.0:
        raise ValueError("no phase separation for G * rho_hi <= 1")
    f = lambda l: np.log(h / l) - G * (h - l)
    return brentq(f, 1e-300, 1.0 / G, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)


def positions(box):
    """Node coordinates measured from the box centre, shaped [z, y, x, 3]."""
    Lx, Ly, Lz = box
    x = np.arange(Lx) - 0.5 * (Lx - 1)
    y = np.arange(Ly) - 0.5 * (Ly - 1)
    z = np.arange(Lz) - 0.5 * (Lz - 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def velocity_error_E0(u, A, box):
    """Eq. 16: rms of (v - A x) over the box, divided by the rms of A x."""
    A = np.asarray(A, dtype=np.float64).reshape(3, 3)
    v0 = positions(box) @ A.T
    num = np.sqrt(np.mean(np.sum((u - v0) ** 2, axis=-1)))
    den = np.sqrt(np.mean(np.sum(v0 ** 2, axis=-1)))
    return num / den


def phase_field(rho_a, rho_b):
    """phi = (rho_A - rho_B) / (rho_A + rho_B)."""
    return (rho_a - rho_b) / (rho_a + rho_b)


def surface_deformation(rho_a, rho_b):
    """(D_LBM, Omega, V) of Eq. 17 for density fields [z, y, x] (see the module notes)."""
    phi = phase_field(np.asarray(rho_a, dtype=np.float64), np.asarray(rho_b, dtype=np.float64))
    lo, hi = float(phi.min()), float(phi.max())
    span = hi - lo
    # central differences at interior nodes
    gz = 0.5 * (phi[2:, 1:-1, 1:-1] - phi[:-2, 1:-1, 1:-1])
    gy = 0.5 * (phi[1:-1, 2:, 1:-1] - phi[1:-1, :-2, 1:-1])
    gx = 0.5 * (phi[1:-1, 1:-1, 2:] - phi[1:-1, 1:-1, :-2])
    area = float(np.sum(np.sqrt(gx * gx + gy * gy + gz * gz))) / span
    volume = float(np.sum(phi - lo)) / span
    area0 = (36.0 * np.pi * volume * volume) ** (1.0 / 3.0)
    return float(np.sqrt(max(0.0, 1.0 - area0 / area))), area, volume


def reinject_mass(f, target):
    """Populations f [2, 19, z, y, x] with the droplet component (0) scaled by
    one factor at the nodes where phi > 0, so that its total mass is target."""
    f = np.array(f, dtype=np.float64)
    ra, rb = f[0].sum(axis=0), f[1].sum(axis=0)
    inside = phase_field(ra, rb) > 0.0
    m_in, m_out = float(ra[inside].sum()), float(ra[~inside].sum())
    k = (target - m_out) / m_in
    f[0][:, inside] *= k
    return f
