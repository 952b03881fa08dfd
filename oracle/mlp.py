"""ORACLE -- test infrastructure only.

Plain float64 multilayer perceptron of the learned surrogate: the reference
for the GPU forward pass and gradients.  The surrogate is an addition of this
library beside the paper's method: it maps a window of the velocity gradient
A(t) to the conformation tensor M of the droplet, whose shape the paper
describes through the Maffettone-Minale tensor of Sec. 2 (Eqs. 1, 2, 5).

Model (layer sizes d0 -> d1 -> ... -> dL):
    x_hat = (x - x_mean) * x_scale                 input normalisation
    h_0 = x_hat
    z_l = h_{l-1} W_l^T + b_l,  h_l = max(z_l, 0)  hidden layers l = 1 .. L-1
    y_hat = h_{L-1} W_L^T + b_L                     normalised output
    y = y_hat / y_scale + y_mean                    output in physical units
Loss on a batch of n samples with targets t:
    t_hat = (t - y_mean) * y_scale
    loss = sum((y_hat - t_hat)^2) / (n * d_L)
W_l has shape (d_l, d_{l-1}), b_l shape (d_l,).

``rounding`` optionally rounds, as the GPU kernels do, to bfloat16 at the
points where they store 16-bit values: the normalised input, the weights,
every hidden activation and every gradient fed to a matrix product.
"""

import numpy as np


def bf16(a):
    """Round float64 values to bfloat16 (nearest even), via float32."""
    a32 = np.asarray(a, dtype=np.float64).astype(np.float32)
    b = a32.view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


class MLP:
    def __init__(self, sizes, params=None, seed=0):
        self.sizes = tuple(int(v) for v in sizes)
        if params is None:
            rng = np.random.default_rng(seed)
            params = []
            for d_in, d_out in zip(self.sizes[:-1], self.sizes[1:]):
                params.append(rng.normal(0.0, np.sqrt(2.0 / d_in), (d_out, d_in)))
                params.append(np.zeros(d_out))
        self.params = [np.array(p, dtype=np.float64) for p in params]
        self.x_mean = np.zeros(self.sizes[0])
        self.x_scale = np.ones(self.sizes[0])
        self.y_mean = np.zeros(self.sizes[-1])
        self.y_scale = np.ones(self.sizes[-1])

    @property
    def layers(self):
        return len(self.sizes) - 1

    def _forward(self, x, rounding):
        r = bf16 if rounding else (lambda a: a)
        h = r((np.asarray(x, dtype=np.float64) - self.x_mean) * self.x_scale)
        hs = [h]
        for l in range(self.layers):
            W, b = r(self.params[2 * l]), self.params[2 * l + 1]
            z = h @ W.T + b
            if l < self.layers - 1:
                h = r(np.maximum(z, 0.0))
                hs.append(h)
            else:
                y_hat = z
        return hs, y_hat

    def forward(self, x, rounding=False):
        """Outputs y in physical units for inputs x of shape (n, d0)."""
        _, y_hat = self._forward(x, rounding)
        return y_hat / self.y_scale + self.y_mean

    def loss_and_gradients(self, x, t, rounding=False):
        """(loss, [dW_1, db_1, ..., dW_L, db_L]) for inputs x and targets t."""
        r = bf16 if rounding else (lambda a: a)
        hs, y_hat = self._forward(x, rounding)
        n = y_hat.shape[0]
        t_hat = (np.asarray(t, dtype=np.float64) - self.y_mean) * self.y_scale
        diff = y_hat - t_hat
        loss = float(np.sum(diff * diff) / (n * self.sizes[-1]))
        g = r(2.0 * diff / (n * self.sizes[-1]))  # d loss / d z_L
        grads = [None] * (2 * self.layers)
        for l in range(self.layers - 1, -1, -1):
            grads[2 * l] = g.T @ hs[l]
            grads[2 * l + 1] = g.sum(axis=0)
            if l > 0:
                dh = g @ r(self.params[2 * l])
                g = r(dh * (hs[l] > 0.0))
        return loss, grads
