"""The surrogate's MLP kernels (lbm_mlp_*) against the float64 MLP of oracle/mlp.py.

Tolerances: the GPU stores the normalised input, weights, hidden activations
and back-propagated gradients in bfloat16 (8 significant bits) and
accumulates in float32.
* Against the float64 MLP that rounds to bfloat16 at the same points: the
  float32 accumulation moves a pre-activation by about 1e-6 relative, which
  can send a bfloat16 rounding the other way (one step of 2^-8) in a few
  values per thousand; outputs agree to 3e-3 of their largest magnitude,
  gradients to 2e-2 in relative L2 norm per layer and, element by element,
  to 3e-2 of the layer's largest gradient entry.
* Against the plain float64 MLP (no rounding): bfloat16 storage alone moves
  outputs and gradients by about 2^-9 relative per stored operand, a few
  times over through the layers: 3e-2 (outputs), 8e-2 (gradients), with each
  layer's gradient direction within cos >= 0.995.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIZES = (576, 256, 256, 256, 6)


@pytest.fixture(scope="session")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


def _cpu_model(net, sizes, norm):
    from oracle.mlp import MLP as CPU

    flat = net.get_params().astype(np.float64)
    params, o = [], 0
    for d_in, d_out in zip(sizes[:-1], sizes[1:]):
        params.append(flat[o:o + d_in * d_out].reshape(d_out, d_in))
        o += d_in * d_out
        params.append(flat[o:o + d_out])
        o += d_out
    cpu = CPU(sizes, params=params)
    cpu.x_mean, cpu.x_scale, cpu.y_mean, cpu.y_scale = [np.asarray(v, dtype=np.float32).astype(np.float64)
                                                        for v in norm]
    return cpu


def _setup(n, seed):
    import torch

    from paper_2112_09972_gb300.lbm import MLP

    rng = np.random.default_rng(seed)
    net = MLP(SIZES, max_batch=max(256, n), seed=seed)
    # non-zero biases, and a normalisation that matters
    p = net.get_params()
    p += rng.normal(0.0, 0.05, p.shape).astype(np.float32)
    net.set_params(p)
    norm = (rng.normal(0.0, 0.01, SIZES[0]), rng.uniform(50.0, 150.0, SIZES[0]), rng.normal(1.0, 0.1, 6),
            rng.uniform(5.0, 20.0, 6))
    net.set_normalisation(*norm)
    x = rng.normal(0.0, 0.01, (n, SIZES[0])).astype(np.float32)
    t = (norm[2] + rng.normal(0.0, 0.1, (n, 6))).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    return net, norm, x, t, xd, td


def test_forward_matches_float64(built):
    import torch

    n = 200  # not a multiple of the 64-row tile
    net, norm, x, _, xd, _ = _setup(n, 1)
    y = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    net.sync()
    cpu = _cpu_model(net, SIZES, norm)
    ref_r = cpu.forward(x, rounding=True)
    ref = cpu.forward(x)
    # compare normalised outputs (the physical ones add a large mean)
    s = np.asarray(norm[3], dtype=np.float64)
    yn = (y.cpu().numpy() - norm[2]) * s
    rn_r = (ref_r - norm[2]) * s
    rn = (ref - norm[2]) * s
    assert np.max(np.abs(yn - rn_r)) <= 3e-3 * np.max(np.abs(rn_r))
    assert np.max(np.abs(yn - rn)) <= 3e-2 * np.max(np.abs(rn))


def test_forward_many_tiles_per_cta(built):
    """Batch 20,480: 320 output tiles of the hidden layers on at most one CTA
    per SM, so each persistent CTA takes two or three tiles (its stage ring
    and both tensor-memory accumulators wrap).  Every row against the
    mma.sync path, and 512 sampled rows against the float64 MLP that rounds
    at the same points."""
    import torch

    n = 20480
    net, norm, x, _, xd, _ = _setup(n, 6)
    outs = []
    for path in (0, 1):
        net.set_tensor_path(path)
        y = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        net.forward(xd, y)
        net.sync()
        outs.append((y.cpu().numpy().astype(np.float64) - norm[2]) * np.asarray(norm[3], dtype=np.float64))
    y0, y1 = outs
    assert np.max(np.abs(y0 - y1)) <= 1e-2 * np.max(np.abs(y1))
    rows = np.random.default_rng(3).choice(n, 512, replace=False)
    cpu = _cpu_model(net, SIZES, norm)
    ref = (cpu.forward(x[rows], rounding=True) - norm[2]) * np.asarray(norm[3], dtype=np.float64)
    assert np.max(np.abs(y0[rows] - ref)) <= 3e-3 * np.max(np.abs(ref))


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n", [128, 4096])
def test_gradients_match_float64(built, n, path):
    """n = 4096: the weight gradients (K = n) are cut into K slices whose
    float32 partials are added in order, on either tensor path, and the bias
    gradients sum 16 row slices."""
    net, norm, x, t, xd, td = _setup(n, 2)
    net.set_tensor_path(path)
    loss, g = net.gradients(xd, td)
    cpu = _cpu_model(net, SIZES, norm)
    loss_r, gr = cpu.loss_and_gradients(x, t, rounding=True)
    loss_p, gp = cpu.loss_and_gradients(x, t)
    assert abs(loss - loss_r) <= 1e-3 * loss_r
    assert abs(loss - loss_p) <= 1e-2 * loss_p
    o = 0
    for k, (ar, ap) in enumerate(zip(gr, gp)):
        gk = g[o:o + ar.size].astype(np.float64).reshape(ar.shape)
        o += ar.size
        assert np.linalg.norm(gk - ar) <= 2e-2 * np.linalg.norm(ar), ("rounded", k)
        assert np.linalg.norm(gk - ap) <= 8e-2 * np.linalg.norm(ap), ("plain", k)
        # element by element: every gradient entry within a fraction of the
        # layer's largest entry of the float64 model that rounds to bfloat16
        # at the same points (a flipped bfloat16 rounding of one stored
        # activation moves the entries it feeds by 2^-8 of that activation)
        err = float(np.max(np.abs(gk - ar)) / np.max(np.abs(ar)))
        assert err <= 3e-2, ("element-wise", k, err)
        cos = float(np.sum(gk * ap) / (np.linalg.norm(gk) * np.linalg.norm(ap)))
        assert cos >= 0.995, (k, cos)
    assert o == g.size


def test_training_fits_a_smooth_map(built):
    """A smooth nonlinear map of a 576-vector to 6 outputs: Adam on the GPU
    lowers the loss by more than 10x within 600 steps."""
    import torch

    from paper_2112_09972_gb300.lbm import MLP

    rng = np.random.default_rng(5)
    n = 8192
    x = rng.normal(0.0, 1.0, (n, 576)).astype(np.float32)
    P = rng.normal(0.0, 1.0 / 24.0, (576, 6))
    t = (np.tanh(x @ P) + 0.3 * (x @ P) ** 2).astype(np.float32)
    net = MLP(SIZES, max_batch=512, seed=7)
    net.set_normalisation(np.zeros(576), np.ones(576), t.mean(0), 1.0 / t.std(0))
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    first = net.gradients(xd[:512].contiguous(), td[:512].contiguous())[0]
    for s in range(600):
        i = (s * 512) % n
        net.train_step(xd[i:i + 512].contiguous(), td[i:i + 512].contiguous(), 1e-3)
    last = net.gradients(xd[:512].contiguous(), td[:512].contiguous())[0]
    assert last < first / 10.0, (first, last)


def test_deformation_of_predicted_m(built):
    """D of Eq. 4 from M's eigenvalues, against numpy's eigh, on symmetric
    positive definite matrices written into the network's output path."""
    import torch

    from paper_2112_09972_gb300.lbm import MLP

    rng = np.random.default_rng(9)
    n = 300
    # a network whose output is its last bias: zero weights, y = b / scale + mean
    net = MLP((32, 32, 6), max_batch=64, seed=0)
    Ms = []
    for _ in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = rng.uniform(0.5, 2.0, 3)
        Ms.append(Q @ np.diag(lam) @ Q.T)
    Ms = np.array(Ms)
    m6 = np.stack([Ms[:, 0, 0], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 1], Ms[:, 1, 2], Ms[:, 2, 2]], axis=1)
    D = torch.empty(n, dtype=torch.float64, device="cuda")
    out = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    params = np.zeros(net.param_count(), dtype=np.float32)
    x = torch.zeros((1, 32), dtype=torch.float32, device="cuda")
    for r in range(n):
        # y = y_mean when the output is zero
        net.set_normalisation(np.zeros(32), np.ones(32), m6[r], np.ones(6))
        net.set_params(params)
        net.deformation(x, out[r:r + 1], D[r:r + 1])
    net.sync()
    lam = np.linalg.eigvalsh(out.cpu().numpy().astype(np.float64)[:, [0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(n, 3, 3))
    ref = (np.sqrt(lam[:, 2]) - np.sqrt(lam[:, 0])) / (np.sqrt(lam[:, 2]) + np.sqrt(lam[:, 0]))
    assert np.max(np.abs(D.cpu().numpy() - ref)) <= 1e-12


def test_invalid_shapes_rejected(built):
    from paper_2112_09972_gb300.lbm import MLP, LBMError

    with pytest.raises(LBMError):
        MLP((100, 256, 6), max_batch=64)  # input width not a multiple of 32
    with pytest.raises(LBMError):
        MLP((576, 256, 64), max_batch=64)  # more than 32 outputs
    with pytest.raises(LBMError):
        MLP((576, 256, 6), max_batch=100)  # batch not a multiple of 32


def test_tcgen05_and_mma_sync_paths_agree(built):
    """Batch 256: the forward products (N tiles of 128 and, for the 32-wide
    output layer, 32), the masked back-propagation products and the weight
    gradients (N tile 64 for the 576-wide first layer) run on tcgen05 tensor
    cores by default and on mma.sync with path 1.  Both accumulate bfloat16 products in float32 in a
    different order, so a stored bfloat16 activation can round the other way:
    outputs agree to 1e-2 of their largest magnitude, gradients to 2e-2 in
    relative L2 norm per layer; a wrong operand layout would miss by O(1)."""
    import torch

    n = 256
    net, norm, x, t, xd, td = _setup(n, 4)
    out = {}
    for path in (0, 1):
        net.set_tensor_path(path)
        y = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        net.forward(xd, y)
        net.sync()
        loss, g = net.gradients(xd, td)
        out[path] = ((y.cpu().numpy() - norm[2]) * np.asarray(norm[3]), loss, g)
    y0, l0, g0 = out[0]
    y1, l1, g1 = out[1]
    assert np.max(np.abs(y0 - y1)) <= 1e-2 * np.max(np.abs(y1))
    assert abs(l0 - l1) <= 1e-2 * l1
    o = 0
    for d_in, d_out in zip(SIZES[:-1], SIZES[1:]):
        for size in (d_in * d_out, d_out):
            a, b = g0[o:o + size], g1[o:o + size]
            o += size
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b)
