"""The batched ensemble (lbm_batch_*) against the oracle and the single-box path,
in both of its launch kinds: the generic tile march (a box with Ly not a
multiple of 8 selects it) and the row kernel over rows padded to 64 (every
box Lx <= 64, Ly a multiple of 8; widths below 64 leave idle padding nodes,
one box is a full-width row, and z chunks are ragged)."""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads
from paper_2112_09972_gb300.lbm import BatchLBM, DropletLBM

pytestmark = pytest.mark.gpu

W = workloads.C1_PARITY


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


SETS = {"tile": ([(24, 24, 20), (20, 18, 22), (16, 16, 16)], 0),
        "rows": ([(24, 24, 20), (40, 16, 18), (16, 8, 12), (64, 8, 9)], 1)}


@pytest.fixture(params=["tile", "rows"])
def boxes(request):
    return SETS[request.param]


def _histories(BOXES, nsteps, seed=21):
    """OU gradients of each box rescaled by Eq. 15 to a boundary speed of 0.1 on
    its largest edge (the ensemble's driving): strong enough that a wrong
    frame origin of one box moves its droplet measurably within the test."""
    return np.stack([inputs.rescale_to_lattice(inputs.ou_gradient_history(nsteps, 30.0, 400.0, seed, box_id=k), 0.1,
                                               max(b)) for k, b in enumerate(BOXES)], axis=1)


def test_batch_matches_oracle_per_box(built, oracle_mod, boxes):
    BOXES, kind = boxes
    n = 30
    hist = _histories(BOXES, n)
    R = [min(b) / 5 for b in BOXES]
    bt = BatchLBM(BOXES, R, W.visc, W.G, rho_lo=W.rho_lo, z_chunk=7)
    assert bt.launch_kind() == kind
    bt.set_gradients(hist)
    f0 = []
    for k, box in enumerate(BOXES):
        o = oracle_mod.OracleLBM(box, (W.tau, W.tau), W.G, (W.rho_lo, W.rho_hi))
        o.init_droplet(R[k], W.xi, W.rho_hi, W.rho_lo, hist[0, k])
        f = inputs.perturbed_populations(o.populations(), 1e-3, seed=k)
        bt.set_populations(k, f)
        f0.append(f)
    bt.step(n)
    for k, box in enumerate(BOXES):
        o = oracle_mod.OracleLBM(box, (W.tau, W.tau), W.G, (W.rho_lo, W.rho_hi))
        o.set_populations(f0[k])
        o.run(n, np.arange(n), hist[:, k])
        assert rel_linf(bt.populations(k), o.populations()) <= 2e-5, k


def test_batch_matches_single_box_contexts(built, boxes):
    BOXES, kind = boxes
    n = 41
    hist = _histories(BOXES, n, seed=5)
    R = [min(b) / 5 for b in BOXES]
    bt = BatchLBM(BOXES, R, W.visc, W.G, rho_lo=W.rho_lo)
    assert bt.launch_kind() == kind
    bt.set_gradients(hist)
    bt.step(n)
    D, axes, c = bt.deformation()
    for k, box in enumerate(BOXES):
        g = DropletLBM(box, R[k], W.visc, W.G, precision="fp32", rho_lo=W.rho_lo, tile_y=2)
        g.set_gradient_table(np.arange(n), hist[:, k])
        g.step(n)
        Dk, ak, _, ck = g.deformation()
        assert abs(D[k] - Dk) <= 1e-5 * abs(Dk) + 1e-7
        assert np.allclose(c[k], ck, atol=1e-5)
        assert rel_linf(bt.populations(k), g.populations()) <= 1e-5


def test_batch_graph_replay_is_deterministic(built, boxes):
    BOXES, kind = boxes
    hist = _histories(BOXES, 12, seed=9)
    R = [min(b) / 5 for b in BOXES]
    a = BatchLBM(BOXES, R, W.visc, W.G, rho_lo=W.rho_lo)
    b = BatchLBM(BOXES, R, W.visc, W.G, rho_lo=W.rho_lo)
    a.set_gradients(hist)
    b.set_gradients(hist)
    a.step(9)  # four graph replays and one single step
    for k in (1, 2, 3, 1, 2):
        b.step(k)
    for k in range(len(BOXES)):
        assert np.array_equal(a.populations(k), b.populations(k))


def test_batch_autotune_restores_initial_state(built, boxes):
    BOXES, kind = boxes
    hist = _histories(BOXES, 10, seed=2)
    R = [min(b) / 5 for b in BOXES]
    a = BatchLBM(BOXES, R, W.visc, W.G, rho_lo=W.rho_lo)
    a.set_gradients(hist)
    zc, per = a.autotune(trial_steps=2)
    if kind:
        assert zc in (16, 22, 32, 43, 64) and per == 0
    else:
        assert zc in (8, 16, 32, 64) and per in (0, 2, 4)
    a.step(10)
    b = BatchLBM(BOXES, R, W.visc, W.G, rho_lo=W.rho_lo, z_chunk=zc)
    b.set_gradients(hist)
    b.step(10)
    for k in range(len(BOXES)):
        assert rel_linf(a.populations(k), b.populations(k)) <= 1e-6
