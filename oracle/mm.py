"""Maffettone-Minale ellipsoidal droplet model (test infrastructure only).

Restates Sec. 2 of the paper: the morphology tensor M_ij evolves by Eq. 1,

    dM/dt~ = Ca [ f2 (S~ M + M S~) + Omega~ M - M Omega~ ] - f1 (M - 3 III_M/II_M delta),

with S, Omega the symmetric and antisymmetric parts of G_ij = d_j v_i (Eq. 2),
III_M = det M, II_M = ((tr M)^2 - M:M)/2, and the closure coefficients of
Eq. 5.  Time t~ is measured in units of the droplet time tau_d = eta_s R/sigma,
the gradients S~, Omega~ are normalised by G = ||G_ij||_inf (element-wise
maximum; Eq. 3), so Ca = tau_d G and Ca S~ = tau_d S.  D follows Eq. 4 with the
axes sqrt of the eigenvalues of M.  Integration is classical RK4 in FP64.
"""

import numpy as np


def f1(chi):
    """Eq. 5, first closure coefficient."""
    return 40.0 * (chi + 1.0) / ((3.0 + 2.0 * chi) * (16.0 + 19.0 * chi))


def f2(chi, Ca):
    """Eq. 5, second closure coefficient."""
    return 5.0 / (3.0 + 2.0 * chi) + 3.0 * Ca ** 2 / (2.0 + 6.0 * Ca ** 2)


def invariants(M):
    """(II_M, III_M) as defined under Eq. 2."""
    tr = np.trace(M)
    II = 0.5 * (tr * tr - np.sum(M * M))
    III = np.linalg.det(M)
    return II, III


def rhs(M, Gmat, tau_d, chi):
    """dM/dt~ for the velocity gradient Gmat (lattice units) and droplet time tau_d."""
    Gmat = np.asarray(Gmat, dtype=np.float64).reshape(3, 3)
    S = 0.5 * (Gmat + Gmat.T)
    W = 0.5 * (Gmat - Gmat.T)
    Ca = tau_d * np.max(np.abs(Gmat))
    II, III = invariants(M)
    flow = f2(chi, Ca) * tau_d * (S @ M + M @ S) + tau_d * (W @ M - M @ W)
    relax = f1(chi) * (M - 3.0 * III / II * np.eye(3))
    return flow - relax


def deformation(M):
    """Eq. 4 with L, W the square roots of the extreme eigenvalues of M."""
    lam = np.linalg.eigvalsh(M)
    L = np.sqrt(lam[-1])
    W = np.sqrt(lam[0])
    return (L - W) / (L + W)


def integrate(grad_of_t, t_end, tau_d, chi, h=None, M0=None, record_every=None):
    """RK4 from M0 (default: the sphere, delta) over LBM time [0, t_end].

    ``grad_of_t(t)`` returns the 3x3 gradient at LBM time t.  ``h`` is the
    step in LBM time (default tau_d/200).  Returns (M(t_end), times, D(t)).
    """
    h = tau_d / 200.0 if h is None else float(h)
    M = np.eye(3) if M0 is None else np.array(M0, dtype=np.float64)
    n = max(1, int(np.ceil(t_end / h)))
    h = t_end / n
    times, Ds = [0.0], [deformation(M)]
    for k in range(n):
        t = k * h
        # dM/dt = rhs / tau_d in LBM time.
        k1 = rhs(M, grad_of_t(t), tau_d, chi) / tau_d
        k2 = rhs(M + 0.5 * h * k1, grad_of_t(t + 0.5 * h), tau_d, chi) / tau_d
        k3 = rhs(M + 0.5 * h * k2, grad_of_t(t + 0.5 * h), tau_d, chi) / tau_d
        k4 = rhs(M + h * k3, grad_of_t(t + h), tau_d, chi) / tau_d
        M = M + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        if record_every and (k + 1) % record_every == 0:
            times.append(t + h)
            Ds.append(deformation(M))
    times.append(t_end)
    Ds.append(deformation(M))
    return M, np.array(times), np.array(Ds)
