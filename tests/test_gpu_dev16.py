"""16-bit deviation storage (precisions "fp16dev" / "bf16dev") on the GPU.

References: the FP64 oracle with its storage model (the same storage
rounding, float64 arithmetic) and the plain FP64 oracle (the paper's method).

Tolerances:
* against the storage model, one step from the same state: the GPU collides
  in float32, so a deviation that the oracle rounds one way may round to the
  neighbouring value of the format; each moving population agrees to one
  spacing of the format at its deviation (2^-10 |d| binary16, 2^-7 |d|
  bfloat16; the spacing above |d| (1 + 2^-8), for deviations that sit at a
  power of two) plus float32 rounding (2e-7), and each rest population, which
  closes the node's mass, to the sum of those spacings;
* against the plain oracle after the 2000 steps of the 32^3 parity case: D to
  1e-3 relative (the criterion of the fp32 path), and the fields within three
  times the departure of the storage model itself from the plain oracle
  (measured here on the same run) plus 2e-4.
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads
from paper_2112_09972_gb300.lbm import DropletLBM, LBMError

pytestmark = pytest.mark.gpu

FORMATS = {"fp16dev": (10, -14), "bf16dev": (7, -126)}  # fraction bits, smallest normal exponent


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="session")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


def spacing(d, storage):
    frac, emin = FORMATS[storage]
    a = np.abs(d)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(np.where(a > 0, e, emin), emin)
    return 2.0 ** (e - frac)


def destination_density(f, box, periodic, rho_b):
    """float32 density of the node each population streams to, [2, 19, z, y, x]."""
    Lx, Ly, Lz = box
    rs = f.sum(axis=1).astype(np.float32).astype(np.float64)
    from oracle import lbm as olbm

    c, _ = olbm.lattice()
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    out = np.empty_like(f)
    rb = np.float32(rho_b).astype(np.float64)
    for s in range(2):
        for i in range(19):
            xd, yd, zd = x + c[i, 0], y + c[i, 1], z + c[i, 2]
            if periodic:
                out[s, i] = rs[s][zd % Lz, yd % Ly, xd % Lx]
            else:
                inside = (xd >= 0) & (xd < Lx) & (yd >= 0) & (yd < Ly) & (zd >= 0) & (zd < Lz)
                out[s, i] = np.where(inside, rs[s][np.clip(zd, 0, Lz - 1), np.clip(yd, 0, Ly - 1),
                                                   np.clip(xd, 0, Lx - 1)], rb[s])
    return out


def assert_within_one_spacing(g, o, box, periodic, rho_b, storage, stepped=False):
    from oracle import lbm as olbm

    _, w = olbm.lattice()
    dest = destination_density(o, box, periodic, rho_b)
    d = o - w[None, :, None, None, None] * dest
    sp = spacing(d * (1.0 + 2.0 ** -8), storage)
    if stepped and not periodic:
        # The ghost populations pulled by the outermost layer of nodes are
        # 16-bit deviations too, built in float32 on the GPU: one of them may
        # round to the neighbouring value, which moves that node's density and
        # velocity and so its outputs, by up to one spacing at the largest
        # deviation of the layer; the force (Eq. 7) carries a share of that
        # into the second layer.
        Lx, Ly, Lz = box
        z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
        edge = (x <= 1) | (x >= Lx - 2) | (y <= 1) | (y >= Ly - 2) | (z <= 1) | (z >= Lz - 2)
        sp = sp + np.where(edge, np.max(sp[:, 1:][:, :, edge]), 0.0)[None, None]
    err = np.abs(g - o)
    moving = err[:, 1:] <= sp[:, 1:] + 2e-7
    assert moving.all(), float(np.max(err[:, 1:] - sp[:, 1:]))
    rest_tol = sp[:, 1:].sum(axis=1) + 1e-6
    assert np.all(err[:, 0] <= rest_tol)


def _perturbed(oracle_mod, box, R, periodic, seed):
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), periodic=periodic)
    A = inputs.ou_gradient_history(1, 30.0, 400.0, seed=seed)[0]
    o.init_droplet(R, 1.0, 1.0, workloads.RHO_LO, A)
    return inputs.perturbed_populations(o.populations(), 1e-3, seed=seed), A


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_initial_state_matches_storage_model(built, oracle_mod, storage):
    box = (32, 24, 20)
    A = inputs.simple_shear(0.004)
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), storage=storage)
    o.init_droplet(6.0, 1.0, 1.0, workloads.RHO_LO, A)
    g = DropletLBM(box, 6.0, (0.5 / 3, 0.5 / 3), 3.5, precision=storage, rho_hi=1.0, rho_lo=workloads.RHO_LO)
    g.set_gradient(A, 0)
    assert_within_one_spacing(g.populations(), o.populations(), box, False, (workloads.RHO_LO, 1.0), storage)


# (box, periodic, tile_y, row variant): the row-tiled cluster kernel (widths
# 64 and 256; per-thread loads, bulk-copy staging, loader and collider
# threads) and the generic tile kernel (tile_y > 0, and the periodic mode)
CASES = [((64, 24, 20), False, 0, 1), ((256, 16, 12), False, 0, 1), ((64, 24, 20), False, 0, 2),
         ((256, 16, 12), False, 0, 2), ((64, 24, 20), False, 0, 3), ((256, 16, 12), False, 0, 3),
         ((37, 29, 23), False, 3, 0), ((30, 26, 22), True, 4, 0)]


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
@pytest.mark.parametrize("box,periodic,tile_y,variant", CASES)
def test_one_step_matches_storage_model(built, oracle_mod, storage, box, periodic, tile_y, variant):
    f0, A = _perturbed(oracle_mod, box, 4.0, periodic, seed=3)
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0), periodic=periodic, storage=storage)
    o.set_populations(f0)
    g = DropletLBM(box, 4.0, (0.5 / 3, 0.5 / 3), 3.5, precision=storage, periodic=periodic, rho_hi=1.0,
                   rho_lo=workloads.RHO_LO, tile_y=tile_y, z_chunk=5, row_variant=variant)
    g.set_populations(f0)
    rho_b = (workloads.RHO_LO, 1.0)
    # the upload is the storage model's conversion
    assert_within_one_spacing(g.populations(), o.populations(), box, periodic, rho_b, storage)
    # the same stored state on both sides, then one step
    g.set_populations(o.populations())
    g.set_gradient(A, 0)
    o.step(None if periodic else A)
    g.step(1)
    assert_within_one_spacing(g.populations(), o.populations(), box, periodic, rho_b, storage, stepped=True)


@pytest.fixture(scope="module")
def c1_runs(oracle_mod):
    """The 32^3 parity case on the plain oracle and on its storage models."""
    from oracle.observables import deformation_from_moments

    w = workloads.C1_PARITY
    A = inputs.simple_shear(w.shear_rate())
    out = {"A": A}
    for storage in ("exact", "fp16dev", "bf16dev"):
        o = oracle_mod.OracleLBM((w.box,) * 3, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi), storage=storage)
        o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, A)
        o.run(w.steps, [0.0], [A])
        ra, rb, u = o.fields()
        out[storage] = dict(ra=ra, rb=rb, u=u, D=deformation_from_moments(o.moments())[0], mass=o.checksums()[0])
    return out


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_config1_after_2000_steps(built, c1_runs, storage):
    w = workloads.C1_PARITY
    g = DropletLBM((w.box,) * 3, w.R, w.visc, w.G, precision=storage, rho_hi=w.rho_hi, rho_lo=w.rho_lo, xi=w.xi)
    g.set_gradient(c1_runs["A"], 0)
    g.step(w.steps)
    ra, rb, u = g.fields()
    ex, model = c1_runs["exact"], c1_runs[storage]
    for name, val in (("ra", ra), ("rb", rb), ("u", u)):
        model_err = rel_linf(model[name], ex[name])
        assert rel_linf(val, ex[name]) <= 3.0 * model_err + 2e-4, (name, rel_linf(val, ex[name]), model_err)
    D = g.deformation()[0]
    assert abs(D - ex["D"]) <= 1e-3 * abs(ex["D"]) + 1e-6
    assert abs(D - model["D"]) <= 1e-3 * abs(model["D"]) + 1e-6
    mass, _ = g.checksums()
    assert np.allclose(mass, model["mass"], rtol=1e-4)


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_periodic_mass_conserved_to_float32(built, oracle_mod, storage):
    box = (30, 26, 22)
    f0, _ = _perturbed(oracle_mod, box, 5.0, True, seed=6)
    g = DropletLBM(box, 5.0, (0.4 / 3, 0.6 / 3), 3.5, precision=storage, periodic=True, rho_hi=1.0,
                   rho_lo=workloads.RHO_LO)
    g.set_populations(f0)
    m0, p0 = g.checksums()
    g.step(200)
    m1, p1 = g.checksums()
    assert np.all(np.abs(m1 - m0) <= 1e-5 * m0)
    assert np.all(np.abs(p1 - p0) <= 1e-5 * m0.sum())


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_checkpoint_resume_is_bit_identical(built, tmp_path, storage):
    w = workloads.C1_PARITY
    hist = inputs.ou_gradient_history(40, 20.0, 400.0, seed=8)
    mk = lambda: DropletLBM((64, 16, 18), 5.0, w.visc, w.G, precision=storage, rho_lo=w.rho_lo)
    a = mk()
    a.set_gradient_table(np.arange(40), hist)
    a.step(40)
    ref = a.populations()
    b = mk()
    b.set_gradient_table(np.arange(40), hist)
    b.step(15)
    path = tmp_path / "ck.bin"
    b.save(path)
    c = mk()
    c.load(path)
    assert c.step_count() == 15
    c.step(25)
    assert np.array_equal(c.populations(), ref)


@pytest.fixture(scope="module")
def downscaled_model_error(oracle_mod):
    """Departure of the storage model from the exact oracle after ten steps of
    the 64^3, R = 8 downscale of the 256^3 precision case (the same boundary
    speed u_LBM, so the same size of ghost deviations): rel L-inf of rho_A,
    rho_B, u for each format."""
    w = workloads.C4_DOWNSCALED
    box = (w.box,) * 3
    hist = w.gradient_history(10)
    fields = {}
    for storage in ("exact", "fp16dev", "bf16dev"):
        o = oracle_mod.OracleLBM(box, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi), storage=storage)
        o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, hist[0])
        o.run(10, np.arange(10), hist)
        fields[storage] = o.fields()
    return {s: [rel_linf(fields[s][k], fields["exact"][k]) for k in range(3)] for s in ("fp16dev", "bf16dev")}


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_full_size_256_against_fp32(built, downscaled_model_error, storage):
    """The 256^3, R = 32 precision case in the benchmark's launch shape: ten
    steps of 16-bit deviation storage against float32 storage from the same
    initial state.  The departure is the storage rounding, which the ghost
    speed sets: each field within three times the storage model's departure
    on the 64^3 downscale (plus 1e-5; the 256^3 box has 16 times as many
    boundary nodes over which the maximum is taken).  The float32 row kernel at this width is
    checked against the oracle in test_fp32_256_wide_against_oracle."""
    w = workloads.C4_PRECISION
    box = (w.box,) * 3
    hist = w.gradient_history(10)
    runs = {}
    for prec in ("fp32", storage):
        g = DropletLBM(box, w.R, w.visc, w.G, precision=prec, rho_hi=w.rho_hi, rho_lo=w.rho_lo)
        g.set_gradient_table(np.arange(10), hist)
        g.step(10)
        runs[prec] = g.fields() + (g.deformation()[0],)
        g.close()
    a, b = runs["fp32"], runs[storage]
    for k in range(3):
        assert rel_linf(b[k], a[k]) <= 3.0 * downscaled_model_error[storage][k] + 1e-5, k
    assert abs(b[3] - a[3]) <= 1e-3 * abs(a[3]) + 1e-6


@pytest.fixture(scope="module")
def downscale_oracle(oracle_mod):
    """The 64^3, R = 8 downscale of the precision case (its gradient history
    rescaled to the box) on the FP64 oracle: 400 steps from the tanh droplet."""
    from oracle.observables import deformation_from_moments

    w = workloads.C4_DOWNSCALED
    box = (w.box,) * 3
    hist = w.gradient_history(401)
    o = oracle_mod.OracleLBM(box, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi))
    o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, hist[0])
    o.run(400, np.arange(401), hist)
    D, axes, _, _ = deformation_from_moments(o.moments())
    return dict(hist=hist, fields=o.fields(), D=D, axes=axes)


@pytest.mark.parametrize("storage,tol_field,tol_D", [("fp32", 1e-4, 1e-3), ("fp16dev", 2e-3, 1e-3),
                                                     ("bf16dev", 1.5e-2, 1e-2)])
def test_precision_downscale_against_fp64_oracle(built, downscale_oracle, storage, tol_field, tol_D):
    """Every storage form of the precision case against the FP64 oracle on its
    64^3 downscale after 400 steps (the comparison the benchmark's precision
    leg reports): densities and velocity element by element (relative L-inf),
    and D.  binary16 keeps 11 significant bits of each deviation, bfloat16 8:
    the bfloat16 tolerances are 2^3 times wider."""
    w = workloads.C4_DOWNSCALED
    box = (w.box,) * 3
    ref = downscale_oracle
    g = DropletLBM(box, w.R, w.visc, w.G, precision=storage, rho_hi=w.rho_hi, rho_lo=w.rho_lo, xi=w.xi)
    g.set_gradient_table(np.arange(401), ref["hist"])
    g.step(400)
    ra, rb, u = g.fields()
    D, axes, _, _ = g.deformation()
    g.close()
    ora, orb, ou = ref["fields"]
    errs = (rel_linf(ra, ora), rel_linf(rb, orb), rel_linf(u, ou))
    assert errs[0] <= tol_field and errs[1] <= tol_field and errs[2] <= 10 * tol_field, errs
    rel_D = abs(D - ref["D"]) / abs(ref["D"])
    assert rel_D <= tol_D, rel_D


def test_fp32_256_wide_against_oracle(built, oracle_mod):
    box = (256, 16, 12)
    f0, A = _perturbed(oracle_mod, box, 4.0, False, seed=12)
    o = oracle_mod.OracleLBM(box, (1.0, 1.0), 3.5, (workloads.RHO_LO, 1.0))
    o.set_populations(f0)
    g = DropletLBM(box, 4.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp32", rho_hi=1.0, rho_lo=workloads.RHO_LO,
                   z_chunk=5)
    g.set_populations(f0)
    g.set_gradient(A, 0)
    o.run(6, [0.0], [A])
    g.step(6)
    assert rel_linf(g.populations(), o.populations()) <= 1e-5


def test_non_finite_upload_rejected_on_host(built):
    g = DropletLBM((32, 24, 20), 4.0, (0.5 / 3, 0.5 / 3), 3.5, precision="fp16dev", rho_lo=workloads.RHO_LO)
    f = g.populations()
    f[1, 7, 3, 4, 5] = np.inf
    with pytest.raises(LBMError) as e:
        g.set_populations(f)
    assert e.value.code == -1
