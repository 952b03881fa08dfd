"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the method itself: it only draws the
velocity-gradient histories A(t) that drive the boundary, and seeded
population states used as test inputs.  It imports neither the oracle nor the
CUDA library.

The paper drives its boundary with velocity gradients recorded along tracer
trajectories of a pseudo-spectral DNS at Re_lambda = 420 (Sec. 3).  Those data
are not available here; a synthetic stand-in with the statistics of isotropic
turbulence replaces them:

* 8 independent unit-variance Ornstein-Uhlenbeck processes a_k with the exact
  discrete update a <- a e^(-1/T) + sqrt(1 - e^(-2/T)) xi, T the correlation
  time in steps, xi ~ N(0, 1) drawn from numpy's Philox generator keyed by
  (seed, box id);
* A = sum_k s_k a_k B_k over a Frobenius-orthonormal basis of traceless 3x3
  matrices: 5 symmetric (strain) and 3 antisymmetric (rotation) members, so A
  is traceless by construction;
* s_sym = 1/(tau_eta sqrt(10)), s_anti = 1/(tau_eta sqrt(6)), which gives
  <S:S> = <W:W> = 1/(2 tau_eta^2) as in isotropic turbulence and
  <||A||_F^2> tau_eta^2 = 1.
"""

import numpy as np

_R2 = np.sqrt(2.0)
_R6 = np.sqrt(6.0)


def traceless_basis():
    """The 8 Frobenius-orthonormal traceless basis matrices (5 symmetric, 3 antisymmetric)."""
    B = np.zeros((8, 3, 3))
    B[0] = np.diag([1.0, -1.0, 0.0]) / _R2
    B[1] = np.diag([1.0, 1.0, -2.0]) / _R6
    for k, (a, b) in enumerate([(0, 1), (0, 2), (1, 2)]):
        B[2 + k, a, b] = B[2 + k, b, a] = 1.0 / _R2
        B[5 + k, a, b] = 1.0 / _R2
        B[5 + k, b, a] = -1.0 / _R2
    return B


def ou_gradient_history(n_steps, T_corr, tau_eta, seed, box_id=0):
    """Per-step traceless gradients A(t), t = 0..n_steps-1, shaped [n_steps, 9] (row-major)."""
    rng = np.random.Generator(np.random.Philox(key=[int(seed), int(box_id)]))
    decay = np.exp(-1.0 / T_corr)
    kick = np.sqrt(1.0 - np.exp(-2.0 / T_corr))
    xi = rng.standard_normal((n_steps, 8))
    a = np.empty((n_steps, 8))
    a[0] = xi[0]
    for t in range(1, n_steps):
        a[t] = a[t - 1] * decay + kick * xi[t]
    scale = np.array([1.0 / (tau_eta * np.sqrt(10.0))] * 5 + [1.0 / (tau_eta * np.sqrt(6.0))] * 3)
    A = np.einsum("tk,kab->tab", a * scale, traceless_basis())
    return A.reshape(n_steps, 9)


def ou_final_windows(n_traj, n_steps, T_corr, tau_eta, seed, window, stride, u_lbm, L, n_full=0):
    """Many OU gradient histories at once, without storing them whole.

    The same process as ou_gradient_history (8 exact-update OU components on
    the traceless basis), all trajectories driven by one Philox stream keyed
    [seed, 2^32] (a different stream from the per-box histories), each
    rescaled by Eq. 15 with its own maximum.  Returns (W, H): W [n_traj,
    window, 9], the rescaled gradients of steps n_steps - 1 - stride (window -
    1), ..., n_steps - 1 of every trajectory, and H [n_steps, n_full, 9], the
    whole rescaled histories of the first n_full trajectories.
    """
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 1 << 32]))
    decay = np.exp(-1.0 / T_corr)
    kick = np.sqrt(1.0 - np.exp(-2.0 / T_corr))
    scale = np.array([1.0 / (tau_eta * np.sqrt(10.0))] * 5 + [1.0 / (tau_eta * np.sqrt(6.0))] * 3)
    B = (traceless_basis() * scale[:, None, None]).reshape(8, 9)
    rows = n_steps - 1 - stride * np.arange(window - 1, -1, -1)
    slot = {int(r): j for j, r in enumerate(rows)}
    W = np.empty((n_traj, window, 9))
    H = np.empty((n_steps, n_full, 9))
    amax = np.zeros(n_traj)
    a = rng.standard_normal((n_traj, 8))
    for t in range(n_steps):
        if t > 0:
            a = a * decay + kick * rng.standard_normal((n_traj, 8))
        A = a @ B
        amax = np.maximum(amax, np.max(np.abs(A), axis=1))
        if t in slot:
            W[:, slot[t]] = A
        if n_full:
            H[t] = A[:n_full]
    f = float(u_lbm) / (float(L) * amax)
    return W * f[:, None, None], H * f[None, :n_full, None]


def simple_shear(gamma_dot):
    """A = gamma_dot e_x e_y^T, i.e. u_x = gamma_dot * y."""
    A = np.zeros(9)
    A[1] = float(gamma_dot)
    return A


def rescale_to_lattice(G_hist, u_lbm, L):
    """Sec. 4, Eq. 15: G -> u_LBM / (L ||G||_inf) G.

    ||G||_inf is read as the element-wise maximum over the whole trajectory
    (a constant), so the rescaled signal keeps its time dependence.
    """
    G = np.asarray(G_hist, dtype=np.float64)
    return G * (float(u_lbm) / (float(L) * np.max(np.abs(G))))


def perturbed_populations(f, eps, seed):
    """f * (1 + eps * U(-1, 1)), a seeded perturbation of a population array."""
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 7]))
    f = np.asarray(f, dtype=np.float64)
    return f * (1.0 + eps * rng.uniform(-1.0, 1.0, size=f.shape))
