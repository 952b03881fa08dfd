"""Pins of the float64 MLP that the GPU surrogate kernels are checked against.

* forward pass of a hand-sized network against values worked out by hand;
* gradients against central finite differences of the loss (float64);
* normalisation: the loss is taken on normalised outputs, and the forward
  pass returns physical units;
* the bfloat16 rounding equals the bit-level definition of the format.
"""

import numpy as np


def test_forward_by_hand():
    from oracle.mlp import MLP

    # 2 -> 2 -> 1: h = relu([[1, -1], [2, 0.5]] x + [0, -1]), y = [3, -2] h + 0.5
    m = MLP((2, 2, 1), params=[np.array([[1.0, -1.0], [2.0, 0.5]]), np.array([0.0, -1.0]),
                                np.array([[3.0, -2.0]]), np.array([0.5])])
    x = np.array([[1.0, 2.0], [2.0, 0.0]])
    # sample 1: z = (-1, 2.0) -> h = (0, 2) -> y = -4 + 0.5 = -3.5
    # sample 2: z = (2, 3.0)  -> h = (2, 3) -> y = 6 - 6 + 0.5 = 0.5
    assert np.allclose(m.forward(x), [[-3.5], [0.5]], rtol=0, atol=1e-15)
    m.y_mean[:] = 1.0
    m.y_scale[:] = 4.0
    assert np.allclose(m.forward(x), [[1.0 - 3.5 / 4.0], [1.0 + 0.5 / 4.0]], rtol=0, atol=1e-15)


def test_gradients_match_finite_differences():
    from oracle.mlp import MLP

    rng = np.random.default_rng(3)
    m = MLP((7, 6, 5, 3), seed=4)
    for p in m.params[1::2]:
        p[:] = rng.normal(0.0, 0.3, p.shape)
    m.x_mean = rng.normal(0.0, 1.0, 7)
    m.x_scale = rng.uniform(0.5, 2.0, 7)
    m.y_mean = rng.normal(0.0, 1.0, 3)
    m.y_scale = rng.uniform(0.5, 2.0, 3)
    x = rng.normal(0.0, 1.0, (11, 7))
    t = rng.normal(0.0, 1.0, (11, 3))
    _, grads = m.loss_and_gradients(x, t)
    eps = 1e-6
    for k, p in enumerate(m.params):
        num = np.zeros_like(p)
        for idx in np.ndindex(p.shape):
            old = p[idx]
            p[idx] = old + eps
            lp, _ = m.loss_and_gradients(x, t)
            p[idx] = old - eps
            lm, _ = m.loss_and_gradients(x, t)
            p[idx] = old
            num[idx] = (lp - lm) / (2 * eps)
        assert np.max(np.abs(num - grads[k])) <= 1e-7 * max(1.0, np.max(np.abs(num))), k


def test_bf16_rounding_is_the_bit_definition():
    from oracle.mlp import bf16

    # exact bfloat16 values stay; halfway cases go to the even neighbour
    assert bf16(1.0) == 1.0 and bf16(-3.5) == -3.5
    one_plus = 1.0 + 2.0 ** -7  # next bfloat16 above 1
    assert bf16(1.0 + 2.0 ** -8) == 1.0  # tie -> even (1.0)
    assert bf16(one_plus + 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (mantissa ...10)
    assert bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == one_plus
