"""Host-side pieces of the surrogate (paper_2112_09972_gb300/surrogate.py),
on the CPU: the gradient windows, the conformation tensor M from the ten
moments, and the Eq. 15 rescaling of the training histories."""

import numpy as np
import pytest

from paper_2112_09972_gb300 import surrogate


def test_windows_hold_every_stride_th_gradient_oldest_first():
    T, nbox, W, S = 400, 3, 64, 4
    hist = np.arange(T * nbox * 9, dtype=np.float64).reshape(T, nbox, 9)
    t = 300
    win = surrogate.windows_at(hist, t, W, S)
    assert win.shape == (nbox, 9 * W) and win.dtype == np.float32
    for k in range(nbox):
        rows = win[k].reshape(W, 9)
        # the last sample is step t - 1, the first t - 1 - S (W - 1)
        assert np.array_equal(rows[-1], hist[t - 1, k].astype(np.float32))
        assert np.array_equal(rows[0], hist[t - 1 - S * (W - 1), k].astype(np.float32))
        steps = rows[:, 0] // (nbox * 9)  # the step each sample came from (first entry encodes it)
        assert np.array_equal(np.diff(steps), np.full(W - 1, S))


def test_trajectory_windows_are_sample_major():
    hist = np.random.default_rng(1).normal(size=(1200, 5, 9))
    X = surrogate.trajectory_windows(hist, 1024, 8, 6, 64, 4)
    assert X.shape == (6 * 5, 9 * 64)
    for j in range(6):
        assert np.array_equal(X[5 * j:5 * (j + 1)], surrogate.windows_at(hist, 1024 + 8 * (j + 1), 64, 4))


def _moments_of_ellipsoid(a, R=None, centre=(0.0, 0.0, 0.0), mass=7.0):
    """The ten moments of a uniform ellipsoid with semi-axes a along the
    columns of rotation R: I = R diag(a^2 / 5) R^T about the centre."""
    R = np.eye(3) if R is None else R
    c = np.asarray(centre, dtype=np.float64)
    I = R @ np.diag(np.asarray(a, dtype=np.float64) ** 2 / 5.0) @ R.T
    S = I + np.outer(c, c)
    return np.array([mass, *(mass * c), mass * S[0, 0], mass * S[0, 1], mass * S[0, 2], mass * S[1, 1],
                     mass * S[1, 2], mass * S[2, 2]])


def test_conformation_of_a_sphere_is_the_identity():
    M = surrogate.conformation_from_moments(_moments_of_ellipsoid((3.0, 3.0, 3.0), centre=(1.0, -2.0, 0.5)))
    assert np.allclose(M, [1, 0, 0, 1, 0, 1], atol=1e-12)


def test_conformation_matches_the_oracle_and_has_unit_determinant():
    from oracle.observables import conformation_tensor

    rng = np.random.default_rng(4)
    for _ in range(20):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        m = _moments_of_ellipsoid(rng.uniform(2.0, 9.0, 3), Q, rng.normal(size=3), rng.uniform(1.0, 50.0))
        M6 = surrogate.conformation_from_moments(m)
        M = M6[[0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(3, 3)
        assert np.allclose(M, conformation_tensor(m), rtol=1e-12, atol=1e-12)
        assert np.linalg.det(M) == pytest.approx(1.0, rel=1e-12)
    # batched: a stack of moments gives a stack of M
    ms = np.stack([_moments_of_ellipsoid((3.0, 4.0, 5.0)), _moments_of_ellipsoid((2.0, 2.0, 6.0))])
    assert surrogate.conformation_from_moments(ms).shape == (2, 6)


def test_training_histories_reach_the_lattice_speed_of_eq_15():
    edge, u = 40, 0.1
    h = surrogate.gradient_histories(4, 500, edge, seed=9)
    assert h.shape == (500, 4, 9)
    for k in range(4):
        # Eq. 15: the largest element of the rescaled gradient times the box edge is u_LBM
        assert np.max(np.abs(h[:, k])) * edge == pytest.approx(u, rel=1e-12)
        # each box has its own history, and A stays traceless
        assert np.allclose(h[:, k, 0] + h[:, k, 4] + h[:, k, 8], 0.0, atol=1e-15)
    assert not np.allclose(h[:, 0], h[:, 1])
