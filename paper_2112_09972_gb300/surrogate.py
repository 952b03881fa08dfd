"""Learned surrogate of droplet deformation (an addition of this library).

The paper compares its LBM droplets with the Maffettone-Minale model, an ODE
for the droplet's conformation tensor M driven by the velocity gradient along
the trajectory (Sec. 2, Eqs. 1, 2, 5), and names statistics over many
trajectories as its next step (Sec. 6).  The surrogate learns that map from
the LBM itself: a window of W samples of A(t), one every S LBM steps (the
gradient sampling interval of the tracer signal; 9 W inputs), to the six
entries of M = I / det(I)^(1/3), I the central second-moment tensor of the droplet
indicator (Eq. 4).  M is the identity for a sphere, and D follows from M's
eigenvalues exactly as from I's (D does not depend on the normalisation).

Pieces:
* ``lbm_windows``   -- training or reference data from the batched LBM
  (``BatchLBM``): every ``sample_every`` steps after a spin-up, the window of
  the last W gradients of each box and the box's M and D;
* ``Surrogate``     -- the MLP (``lbm.MLP``: bfloat16 tensor-core kernels),
  its normalisation from the training data, training with Adam, and
  prediction of M and D on the GPU;
* ``trajectories_with_fallback`` -- D along whole trajectories from the
  surrogate, re-running on the LBM every trajectory whose predicted D
  exceeds a threshold (0.4: large deformations, where a droplet nears
  breakup, are left to the LBM).

The only host arithmetic is data handling: window slicing, the 3 x 3
conversion of the LBM's moments into M for the training targets, and the
normalisation statistics.
"""

import numpy as np

from . import inputs, workloads
from .lbm import BatchLBM, MLP

WINDOW = 64          # samples of A(t) per input
STRIDE = 4           # LBM steps between samples: the window covers 256 steps, several times the
                     # damping time of the droplet's shape oscillations at tau = 1, R = 8
HIDDEN = (256, 256, 256)
N_OUT = 6            # M_xx, M_xy, M_xz, M_yy, M_yz, M_zz
D_FALLBACK = 0.4     # predicted D above which a trajectory is re-run on the LBM


def conformation_from_moments(m):
    """M = I / det(I)^(1/3) (entries xx, xy, xz, yy, yz, zz) from the ten
    moments [.., 10] of lbm_moments / lbm_batch_moments."""
    m = np.asarray(m, dtype=np.float64)
    mass = m[..., 0]
    c = m[..., 1:4] / mass[..., None]
    I = np.empty(m.shape[:-1] + (3, 3))
    idx = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}
    for (a, b), k in idx.items():
        v = m[..., k] / mass - c[..., a] * c[..., b]
        I[..., a, b] = v
        I[..., b, a] = v
    det = np.linalg.det(I)
    M = I / np.cbrt(det)[..., None, None]
    return np.stack([M[..., 0, 0], M[..., 0, 1], M[..., 0, 2], M[..., 1, 1], M[..., 1, 2], M[..., 2, 2]], axis=-1)


def gradient_histories(nbox, steps, edge, seed, T_corr=200.0, u_lbm=0.1):
    """A[t, k, 9]: one OU history per box (Philox key [seed, k]), rescaled by
    Eq. 15 so that its largest boundary speed on a box of this edge is u_lbm."""
    out = np.empty((steps, nbox, 9))
    for k in range(nbox):
        h = inputs.ou_gradient_history(steps, T_corr, 1.0, seed, box_id=k)
        out[:, k] = inputs.rescale_to_lattice(h, u_lbm, int(edge))
    return out


def windows_at(hist, t, window=WINDOW, stride=STRIDE):
    """Windows ending at step t of every trajectory in hist[t, k, 9]: the
    gradients of steps t - 1 - stride (window - 1), ..., t - 1 - stride, t - 1
    (oldest first), flattened to [nbox, 9 window] float32."""
    rows = t - 1 - stride * np.arange(window - 1, -1, -1)
    return hist[rows].transpose(1, 0, 2).reshape(hist.shape[1], 9 * window).astype(np.float32)


def lbm_windows(hist, edge, spinup, sample_every, nsamples, window=WINDOW, stride=STRIDE, stream=None):
    """Run the batched LBM on boxes of one edge (R = edge / 5) driven by
    hist[t, k, 9]; after `spinup` steps, every `sample_every` steps record for
    each box its window (windows_at), M and D.  Returns (X [n, 9 window]
    float32, M [n, 6] float32, D [n] float64, steps run) with n = nsamples *
    nbox, sample-major."""
    nbox = hist.shape[1]
    total = spinup + sample_every * nsamples
    assert hist.shape[0] >= total and spinup >= stride * window
    bt = BatchLBM([(edge,) * 3] * nbox, [edge / 5.0] * nbox, (1.0 / 6.0, 1.0 / 6.0), workloads.G_COUPLING,
                  rho_lo=workloads.RHO_LO, rho_hi=workloads.RHO_HI, stream=stream)
    bt.set_gradients(hist[:total])
    X, M, D = [], [], []
    bt.step(spinup)
    t = spinup
    for _ in range(nsamples):
        bt.step(sample_every)
        t += sample_every
        m = bt.moments()
        d, _, _ = bt.deformation()
        X.append(windows_at(hist, t, window, stride))
        M.append(conformation_from_moments(m).astype(np.float32))
        D.append(d)
    bt.close()
    return np.concatenate(X), np.concatenate(M), np.concatenate(D), total


class Surrogate:
    """The MLP 9 W -> 256 -> 256 -> 256 -> 6 on the GPU."""

    def __init__(self, window=WINDOW, stride=STRIDE, hidden=HIDDEN, max_batch=16384, seed=0, device=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.window = window
        self.stride = stride
        # one stream for the network's kernels and the torch operations that
        # feed them, so that batches are ordered with the steps that read them
        self.stream = torch.cuda.Stream(device=self.device)
        self.net = MLP((9 * window,) + tuple(hidden) + (N_OUT,), max_batch=max_batch, seed=seed,
                       stream=self.stream.cuda_stream, device=self.device.index)
        self.max_batch = max_batch
        self._copy_stream = torch.cuda.Stream(device=self.device)
        self._staging = None  # two device buffers of max_batch windows (pinned-input pipeline)

    def close(self):
        self.net.close()

    def fit(self, X, Y, steps=2000, batch=512, lr=1e-3, lr_final=1e-5, seed=0, log_every=0):
        """Train on X [n, 9 W], Y [n, 6] (numpy float32) with Adam and a
        geometric learning-rate decay; returns the loss history (every
        log_every steps)."""
        torch = self.torch
        X = np.asarray(X, dtype=np.float32)
        Y = np.asarray(Y, dtype=np.float32)
        x_mean = X.mean(axis=0)
        x_std = X.std(axis=0)
        y_mean = Y.mean(axis=0)
        y_std = Y.std(axis=0)
        self.net.set_normalisation(x_mean, 1.0 / np.maximum(x_std, 1e-12), y_mean, 1.0 / np.maximum(y_std, 1e-12))
        n = X.shape[0]
        decay = (lr_final / lr) ** (1.0 / max(steps - 1, 1))
        hist = []
        with torch.cuda.stream(self.stream):
            Xd = torch.from_numpy(X).to(self.device)
            Yd = torch.from_numpy(Y).to(self.device)
            gen = torch.Generator(device=self.device)
            gen.manual_seed(int(seed))
            perm = torch.randperm(n, device=self.device, generator=gen)
            pos = 0
            for s in range(steps):
                if pos + batch > n:
                    perm = torch.randperm(n, device=self.device, generator=gen)
                    pos = 0
                idx = perm[pos:pos + batch]
                pos += batch
                xb = Xd.index_select(0, idx)
                yb = Yd.index_select(0, idx)
                want = bool(log_every) and (s % log_every == 0 or s == steps - 1)
                loss = self.net.train_step(xb, yb, lr * decay ** s, want_loss=want)
                if want:
                    hist.append((s, loss))
            self.net.sync()
        return hist

    def predict(self, X):
        """(M [n, 6] float32, D [n] float64) of windows X [n, 9 W] (numpy, a
        CPU tensor or a CUDA tensor), as numpy arrays.

        Host windows go to the GPU in chunks of max_batch.  From pinned
        memory the copy of one chunk (on a copy stream, into one of two
        staging buffers) overlaps the forward pass and D of the previous
        chunk; from pageable memory the chunks are copied in turn."""
        torch = self.torch
        n = int(X.shape[0])
        with torch.cuda.stream(self.stream):
            m6 = torch.empty((n, N_OUT), dtype=torch.float32, device=self.device)
            D = torch.empty(n, dtype=torch.float64, device=self.device)
            if isinstance(X, torch.Tensor) and X.is_cuda:
                self.net.deformation(X.contiguous(), m6, D)
            else:
                Xh = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32))
                self._deformation_from_host(Xh.contiguous(), m6, D)
            m6h = torch.empty(m6.shape, dtype=m6.dtype, pin_memory=True)
            Dh = torch.empty(D.shape, dtype=D.dtype, pin_memory=True)
            m6h.copy_(m6, non_blocking=True)
            Dh.copy_(D, non_blocking=True)
            self.net.sync()
            self.stream.synchronize()
        return m6h.numpy(), Dh.numpy()

    def _deformation_from_host(self, Xh, m6, D):
        torch = self.torch
        n, chunk = Xh.shape[0], self.max_batch
        if not Xh.is_pinned():
            for s in range(0, n, chunk):
                e = min(n, s + chunk)
                self.net.deformation(Xh[s:e].to(self.device), m6[s:e], D[s:e])
            return
        if self._staging is None:
            self._staging = [torch.empty((chunk, Xh.shape[1]), dtype=torch.float32, device=self.device)
                             for _ in range(2)]
        done = [None, None]  # the network's stream is through with staging buffer b
        for k, s in enumerate(range(0, n, chunk)):
            e, b = min(n, s + chunk), k % 2
            buf = self._staging[b][:e - s]
            with torch.cuda.stream(self._copy_stream):
                if done[b] is not None:
                    self._copy_stream.wait_event(done[b])
                buf.copy_(Xh[s:e], non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(self._copy_stream)
            self.stream.wait_event(ready)
            self.net.deformation(buf, m6[s:e], D[s:e])
            done[b] = torch.cuda.Event()
            done[b].record(self.stream)


def trajectory_windows(hist, spinup, sample_every, nsamples, window=WINDOW, stride=STRIDE):
    """Windows of every box at the sampling times of lbm_windows, [nsamples * nbox, 9 W]."""
    return np.concatenate([windows_at(hist, spinup + sample_every * (j + 1), window, stride) for j in range(nsamples)])


def trajectories_with_fallback(sur, hist, edge, spinup, sample_every, nsamples, threshold=D_FALLBACK, stream=None):
    """D at every sampling time of every trajectory in hist[t, k, 9]: the
    surrogate's, except for trajectories whose predicted D exceeds
    `threshold` at some sample, which are re-run on the LBM.  Returns
    (D [nsamples, nbox], fallback mask [nbox])."""
    nbox = hist.shape[1]
    X = trajectory_windows(hist, spinup, sample_every, nsamples, sur.window, sur.stride)
    _, D = sur.predict(X)
    D = D.reshape(nsamples, nbox)
    fb = np.any(D > threshold, axis=0)
    if fb.any():
        ks = np.flatnonzero(fb)
        _, _, D_lbm, _ = lbm_windows(hist[:, ks], edge, spinup, sample_every, nsamples, sur.window, sur.stride,
                                     stream)
        D[:, ks] = D_lbm.reshape(nsamples, len(ks))
    return D, fb
