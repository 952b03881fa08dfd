"""Pins of the oracle's storage model (16-bit deviation storage).

The model replaces every stored state by what the format holds: float32
densities rho*, deviations d_i = f_i - w_i rho*(x + c_i) of the moving
populations rounded to binary16 or bfloat16, and a float32 rest population
that closes each node's mass.  The pins check it against definitions that do
not come from the oracle:

* its binary16 and float32 rounding against numpy's IEEE conversions from
  float64 (round to nearest, ties to even, gradual underflow);
* its bfloat16 rounding against the bit-level definition of the format (the
  upper 16 bits of a float32, rounded to nearest-even), on float32 inputs;
* a stored state: densities are the float32 sums of the input, every
  deviation from w_i rho* of the destination node is a value of the format,
  and each node's populations sum to its float32 density;
* dynamics: in the periodic test mode the model conserves each component's
  mass to float32 rounding, and one step departs from the full-precision
  oracle by no more than the format's rounding of the deviations;
* the rest state (uniform ghost densities exact in float32, A = 0) stays a
  fixed point with ghost nodes: bit for bit with binary16 deviations (all
  zero, ghost ones included), and to float32 rounding with bfloat16, whose
  range holds the float32 residues of the rest population.
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads


def _samples(rng, n, lo=-30, hi=3):
    mag = 2.0 ** rng.uniform(lo, hi, n)
    x = np.where(rng.random(n) < 0.5, -mag, mag)
    return x


def test_binary16_rounding_matches_numpy(oracle_mod):
    from oracle import lbm as olbm

    rng = np.random.default_rng(11)
    x = np.concatenate([_samples(rng, 4000), _samples(rng, 500, -26, -14)])  # normal and subnormal range
    # exact ties between two binary16 neighbours: odd multiples of half a spacing
    x = np.concatenate([x, (2 * rng.integers(1, 2000, 200) + 1) * 2.0 ** -12])
    for v in x:
        assert olbm.round_to("binary16", v) == float(np.float16(v)), v


def test_float32_rounding_matches_numpy(oracle_mod):
    from oracle import lbm as olbm

    rng = np.random.default_rng(12)
    for v in np.concatenate([_samples(rng, 3000), _samples(rng, 300, -140, -126)]):
        assert olbm.round_to("float32", v) == float(np.float32(v)), v


def _bf16_by_bits(x32):
    """bfloat16 of float32 values from the bit-level definition."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bfloat16_rounding_matches_bit_definition(oracle_mod):
    from oracle import lbm as olbm

    rng = np.random.default_rng(13)
    x32 = np.concatenate([_samples(rng, 4000), _samples(rng, 300, -140, -126)]).astype(np.float32)
    # ties: a float32 whose low 16 bits are exactly 0x8000
    t = (rng.integers(0x3C000000, 0x40000000, 200, dtype=np.uint64) & 0xFFFF0000) | 0x8000
    x32 = np.concatenate([x32, t.astype(np.uint32).view(np.float32)])
    ref = _bf16_by_bits(x32)
    for v, r in zip(x32.astype(np.float64), ref):
        assert olbm.round_to("bfloat16", v) == r, v


def _state(oracle_mod, box, periodic, seed=5):
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), periodic=periodic)
    A = inputs.ou_gradient_history(1, 50.0, 300.0, seed=seed)[0]
    o.init_droplet(1.6, 1.0, 1.0, workloads.RHO_LO, A)
    return inputs.perturbed_populations(o.populations(), 1e-3, seed=seed)


@pytest.mark.parametrize("storage,fmt", [("fp16dev", np.float16), ("bf16dev", None)])
@pytest.mark.parametrize("periodic", [False, True])
def test_stored_state_is_in_the_format(oracle_mod, storage, fmt, periodic):
    box = (6, 5, 4)
    f = _state(oracle_mod, box, periodic)
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), periodic=periodic, storage=storage)
    o.set_populations(f)
    g = o.populations()
    c, w = oracle_mod.lattice()
    rs = f.sum(axis=1).astype(np.float32).astype(np.float64)  # [2, z, y, x]
    Lx, Ly, Lz = box
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    rho_b = np.float32([workloads.RHO_LO, 1.0]).astype(np.float64)
    for s in range(2):
        for i in range(1, 19):
            xd, yd, zd = x + c[i, 0], y + c[i, 1], z + c[i, 2]
            if periodic:
                dest = rs[s][zd % Lz, yd % Ly, xd % Lx]
            else:
                inside = (xd >= 0) & (xd < Lx) & (yd >= 0) & (yd < Ly) & (zd >= 0) & (zd < Lz)
                dest = np.where(inside, rs[s][np.clip(zd, 0, Lz - 1), np.clip(yd, 0, Ly - 1), np.clip(xd, 0, Lx - 1)],
                                rho_b[s])
            d = g[s, i] - w[i] * dest
            q = np.float16(d).astype(np.float64) if fmt is not None else _bf16_by_bits(d.astype(np.float32))
            assert np.max(np.abs(q - d)) <= 1e-16
            # the stored value stays within the format's rounding of the input
            # deviation: half a spacing, 2^-11 |d| (binary16; 2^-25 in its
            # subnormal range) or 2^-8 |d| (bfloat16)
            rel, sub = (2.0 ** -11, 2.0 ** -25) if fmt is not None else (2.0 ** -8, 2.0 ** -134)
            tol = np.maximum(rel * np.abs(f[s, i] - w[i] * dest), sub) + 1e-15
            assert np.all(np.abs(g[s, i] - f[s, i]) <= tol)
    # each node's populations sum to its float32 density (the rest
    # population is rounded to float32: 2^-24 of its size)
    assert np.max(np.abs(g.sum(axis=1) - rs)) <= 2.0 ** -24 * np.max(np.abs(g[:, 0])) + 1e-15


@pytest.mark.parametrize("storage,ulp", [("fp16dev", 2.0 ** -11), ("bf16dev", 2.0 ** -8)])
def test_storage_dynamics(oracle_mod, storage, ulp):
    box = (8, 7, 6)
    f = _state(oracle_mod, box, True, seed=9)
    ex = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), periodic=True)
    dv = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), periodic=True, storage=storage)
    dv.set_populations(f)
    ex.set_populations(dv.populations())  # the same starting state
    ex.step()
    dv.step()
    # one step: every population within the rounding of its deviation
    # (|d| < 0.05 here) plus float32 rounding of densities
    assert np.max(np.abs(dv.populations() - ex.populations())) <= ulp * 0.05 + 1e-7
    m0 = dv.checksums()[0]
    for _ in range(30):
        dv.step()
    m1 = dv.checksums()[0]
    assert np.all(np.abs(m1 - m0) <= 1e-6 * m0)


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_rest_state_fixed_point_with_ghosts(oracle_mod, storage):
    box = (7, 6, 5)
    # ghost densities exact in float32, so the float64 ghost equilibria and
    # the float32 densities of the state agree exactly
    rho_b = (2.0 ** -9, 1.0)
    o = oracle_mod.OracleLBM(box, (1.0, 1.3), 3.5, rho_b, storage=storage)
    _, w = oracle_mod.lattice()
    f = np.empty(o.shape)
    for s in range(2):
        f[s] = rho_b[s] * w[:, None, None, None]
    o.set_populations(f)
    g0 = o.populations()
    assert np.max(np.abs(g0 - f)) <= 1e-7  # float32 densities
    for _ in range(5):
        o.step(np.zeros(9))
    if storage == "fp16dev":
        assert np.array_equal(o.populations(), g0)
    else:
        # bfloat16 holds residues at the float32 rounding of the rest
        # population (an ulp of 1/3 is 3e-8)
        assert np.max(np.abs(o.populations() - g0)) <= 1e-7
