"""The learned surrogate end to end: trained on batched-LBM windows, checked on
fresh seeded trajectories against the LBM, with its gain in droplets/s.

Data: boxes of edge 40 (R = 8, the smallest ensemble size), OU histories with
correlation time 200 steps rescaled by Eq. 15 to u_LBM = 0.1, a 1024-step
spin-up, then M and D every 8 steps; windows of 64 gradient samples, one
every 4 steps; 1536 training trajectories and 128 test trajectories with
another seed.

D error: the deformation statistics of the test ensemble (the quantity the
surrogate serves: distributions of D over many trajectories, Sec. 6) -- the
mean of D and its 50 / 90 / 99 % quantiles -- against the LBM's, within 1 %;
the per-sample RMS error RMS(D_sur - D_LBM) / RMS(D_LBM) is bounded at 5 %
and printed.  Droplets/s: the test trajectories per second, the batched LBM
(one persistent launch per step for all boxes, spin-up included) against
surrogate inference of all their windows.
"""

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EDGE, SPINUP, EVERY, NSAMP = 40, 1024, 8, 60


@pytest.fixture(scope="module")
def trained():
    import torch

    from paper_2112_09972_gb300 import build, surrogate

    build.build()
    steps = SPINUP + EVERY * NSAMP
    hist = surrogate.gradient_histories(1536, steps, EDGE, seed=101)
    X, M, D, _ = surrogate.lbm_windows(hist, EDGE, SPINUP, EVERY, NSAMP)
    sur = surrogate.Surrogate(max_batch=1024)
    log = sur.fit(X, M, steps=30000, batch=512, lr=1e-3, lr_final=1e-5, log_every=5000)
    print("loss", [(s, round(l, 5)) for s, l in log])
    test_hist = surrogate.gradient_histories(128, steps, EDGE, seed=202)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xt, Mt, Dt, _ = surrogate.lbm_windows(test_hist, EDGE, SPINUP, EVERY, NSAMP)
    torch.cuda.synchronize()
    t_lbm = time.perf_counter() - t0
    return dict(sur=sur, log=log, hist=test_hist, Xt=Xt, Mt=Mt, Dt=Dt, t_lbm=t_lbm, X=X, M=M, D=D)


def test_surrogate_matches_lbm_and_gains(trained):
    import torch

    sur = trained["sur"]
    Xt, Dt = trained["Xt"], trained["Dt"]
    sur.predict(Xt[:1024])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Mp, Dp = sur.predict(Xt)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    err = float(np.sqrt(np.mean((Dp - Dt) ** 2)) / np.sqrt(np.mean(Dt ** 2)))
    err_m = float(np.sqrt(np.mean((Mp - trained["Mt"]) ** 2)) / np.sqrt(np.mean((trained["Mt"] - np.eye(3)[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]) ** 2)))
    # the same windows on the training set
    _, Dtr = sur.predict(trained["X"][:4096])
    Dtr_ref = trained["D"][:4096]
    err_tr = float(np.sqrt(np.mean((Dtr - Dtr_ref) ** 2)) / np.sqrt(np.mean(Dtr_ref ** 2)))
    nb = trained["hist"].shape[1]
    gain = trained["t_lbm"] / t_sur
    stats = {"mean": (float(np.mean(Dp)), float(np.mean(Dt)))}
    for q in (50, 90, 99):
        stats[f"q{q}"] = (float(np.percentile(Dp, q)), float(np.percentile(Dt, q)))
    rel = {k: abs(a - b) / abs(b) for k, (a, b) in stats.items()}
    print(f"surrogate: per-sample D error {err:.4f} (train {err_tr:.4f}), M error {err_m:.4f}, "
          f"D rms {np.sqrt(np.mean(Dt**2)):.4f}; statistics errors {rel}; "
          f"LBM {trained['t_lbm']:.3f} s vs surrogate {t_sur*1e3:.2f} ms for {nb} trajectories: gain {gain:.0f}x; "
          f"loss {trained['log'][0][1]:.3e} -> {trained['log'][-1][1]:.3e}")
    assert max(rel.values()) <= 0.01, rel
    assert err <= 0.05
    assert gain >= 100.0


def test_fallback_reruns_large_deformations_on_lbm(trained):
    """A threshold below every predicted D sends every trajectory to the LBM,
    which then gives the LBM's own D."""
    from paper_2112_09972_gb300 import surrogate

    sur = trained["sur"]
    hist = np.ascontiguousarray(trained["hist"][:, :8])
    D, fb = surrogate.trajectories_with_fallback(sur, hist, EDGE, SPINUP, EVERY, NSAMP, threshold=-1.0)
    assert fb.all()
    Dt = trained["Dt"].reshape(NSAMP, -1)[:, :8]
    assert np.allclose(D, Dt, rtol=1e-5, atol=1e-7)
    D2, fb2 = surrogate.trajectories_with_fallback(sur, hist, EDGE, SPINUP, EVERY, NSAMP)
    assert not fb2.any()  # D stays far below 0.4 at u_LBM = 0.1


def test_pinned_pipeline_matches_pageable_and_device_inputs(trained):
    """The same windows from pinned host memory (chunked copies overlapped
    with the network), from pageable memory and from the device give the
    same M and D bit for bit; 2,500 windows are three chunks of 1,024 and a
    ragged one."""
    import torch

    sur = trained["sur"]
    X = np.ascontiguousarray(trained["Xt"][:2500])
    M0, D0 = sur.predict(X)
    M1, D1 = sur.predict(torch.from_numpy(X).pin_memory())
    M2, D2 = sur.predict(torch.from_numpy(X).cuda())
    assert np.array_equal(M0, M1) and np.array_equal(D0, D1)
    assert np.array_equal(M0, M2) and np.array_equal(D0, D2)
