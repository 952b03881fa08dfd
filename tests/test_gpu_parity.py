"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (float64 oracle as the reference):
* fp64 on the GPU: the same arithmetic in a different order (FMA contraction,
  multiplication by 1/tau instead of division) -- relative L-inf <= 1e-10 on
  fields after 2000 steps, D to 1e-9;
* fp32 on the GPU: rounding of stored populations (2^-24 relative per store)
  accumulated over the run -- relative L-inf <= 1e-4 on rho and u after 2000
  steps, |D_gpu - D_ref| <= 1e-3 |D_ref| + 1e-6.
Relative L-inf is max|a - b| / max|b| over the field.
"""

import os

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads
from paper_2112_09972_gb300.lbm import DropletLBM, LBMError

pytestmark = pytest.mark.gpu


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="session")
def built():
    from paper_2112_09972_gb300 import build

    return build.build()


def _pair(oracle_mod, box, R, tau, G, precision, periodic=False, rho_hi=1.0, rho_lo=workloads.RHO_LO, **kw):
    o = oracle_mod.OracleLBM(box, (tau[0], tau[1]), G, (rho_lo, rho_hi), periodic=periodic)
    visc = ((tau[0] - 0.5) / 3.0, (tau[1] - 0.5) / 3.0)
    g = DropletLBM(box, R, visc, G, precision=precision, periodic=periodic, rho_hi=rho_hi, rho_lo=rho_lo, **kw)
    return o, g


@pytest.fixture(scope="module")
def c1_reference(oracle_mod):
    """Config 1 (32^3, R = 6, simple shear at Ca = 0.1, 2000 steps) on the oracle."""
    w = workloads.C1_PARITY
    A = inputs.simple_shear(w.shear_rate())
    o = oracle_mod.OracleLBM((w.box,) * 3, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi))
    o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, A)
    o.run(w.steps, [0.0], [A])
    from oracle.observables import deformation_from_moments

    D, axes, lam, _ = deformation_from_moments(o.moments())
    ra, rb, u = o.fields()
    return dict(A=A, ra=ra, rb=rb, u=u, D=D, axes=axes, lam=lam, mass=o.checksums()[0])


@pytest.mark.parametrize("precision,tile_y,variant,tol_field,tol_D",
                         [("fp64", 0, 0, 1e-10, 1e-9), ("fp32", 0, 1, 1e-4, 1e-3), ("fp32", 0, 2, 1e-4, 1e-3),
                          ("fp32", 0, 3, 1e-4, 1e-3), ("fp32", 8, 0, 1e-4, 1e-3)])
def test_config1_parity_after_2000_steps(built, c1_reference, precision, tile_y, variant, tol_field, tol_D):
    """fp32 runs every stream-collide kernel: the row-tiled cluster kernel
    (a 32-wide box) with per-thread loads (variant 1), with bulk-copy staging
    (variant 2) and with loader and collider threads (variant 3), and the
    generic tile kernel (tile_y = 8)."""
    w = workloads.C1_PARITY
    g = DropletLBM((w.box,) * 3, w.R, w.visc, w.G, precision=precision, rho_hi=w.rho_hi, rho_lo=w.rho_lo, xi=w.xi,
                   tile_y=tile_y, row_variant=variant)
    g.set_gradient(c1_reference["A"], 0)
    g.step(w.steps)
    ra, rb, u = g.fields()
    assert rel_linf(ra, c1_reference["ra"]) <= tol_field
    assert rel_linf(rb, c1_reference["rb"]) <= tol_field
    assert rel_linf(u, c1_reference["u"]) <= tol_field
    D, axes, lam, _ = g.deformation()
    Dr = c1_reference["D"]
    assert abs(D - Dr) <= tol_D * abs(Dr) + 1e-6
    lr = c1_reference["lam"]
    if (lr[0] - lr[1]) / lr[0] > 1e-3:  # the major axis is unique
        assert abs(axes[:, 0] @ c1_reference["axes"][:, 0]) >= 1 - 1e-3
    assert g.step_count() == w.steps


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("periodic", [False, True])
def test_ragged_box_short_run(built, oracle_mod, precision, tol, periodic):
    """A box that is no multiple of any tile, perturbed state, OU driving."""
    box = (37, 29, 23)
    tau = (0.9, 1.3)
    o, g = _pair(oracle_mod, box, 5.0, tau, 3.5, precision, periodic=periodic, tile_y=3, z_chunk=5)
    hist = inputs.ou_gradient_history(40, 50.0, 300.0, seed=7)
    o.init_droplet(5.0, 1.0, 1.0, workloads.RHO_LO, hist[0])
    f0 = inputs.perturbed_populations(o.populations(), 1e-3, seed=3)
    o.set_populations(f0)
    g.set_populations(f0)
    g.set_gradient_table(np.arange(40), hist)
    for t in range(40):
        o.step(hist[t] if not periodic else None)
    g.step(40)
    assert rel_linf(g.populations(), o.populations()) <= tol
    ra, rb, u = g.fields()
    ora, orb, ou = o.fields()
    assert rel_linf(ra, ora) <= tol and rel_linf(rb, orb) <= tol and rel_linf(u, ou) <= 10 * tol


def test_throughput_case_200_steps_benchmark_launch(built, oracle_mod):
    """The benchmark's own launch -- 128^3, R = 16, fp32, the OU history of the
    throughput case, automatic kernel variant and launch shape (the instance
    bench.py times) -- against the FP64 oracle after 200 steps from the
    same initial state: every stored population, element by element, within
    1e-4 of the largest population, and D within 1e-3.  The run spans every
    CTA of the launch, every march direction and the ghost shell on all six
    faces."""
    from oracle.observables import deformation_from_moments

    w = workloads.C2_THROUGHPUT
    box = (w.box,) * 3
    steps = 200
    hist = w.gradient_history(steps + 1)
    o = oracle_mod.OracleLBM(box, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi))
    o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, hist[0])
    g = DropletLBM(box, w.R, w.visc, w.G, precision=w.precision, rho_hi=w.rho_hi, rho_lo=w.rho_lo, xi=w.xi)
    g.set_populations(o.populations())
    g.set_gradient_table(np.arange(steps + 1), hist)
    g.step(steps)
    o.run(steps, np.arange(steps + 1), hist)
    ref = o.populations()
    assert rel_linf(g.populations(), ref) <= 1e-4
    D_ref = deformation_from_moments(o.moments())[0]
    D = g.deformation()[0]
    assert abs(D - D_ref) <= 1e-3 * abs(D_ref) + 1e-6


def test_interpolated_gradient_knots(built, oracle_mod):
    """Knots every 7 steps, linear interpolation between them (fp64)."""
    box = (12, 14, 10)
    o, g = _pair(oracle_mod, box, 3.0, (1.0, 1.0), 3.5, "fp64")
    kt = np.array([0, 7, 14, 21])
    kA = inputs.ou_gradient_history(4, 3.0, 200.0, seed=2)
    o.init_droplet(3.0, 1.0, 1.0, workloads.RHO_LO, kA[0])
    g.set_gradient_table(kt, kA)
    o.run(25, kt, kA)
    g.step(25)
    assert rel_linf(g.populations(), o.populations()) <= 1e-12


@pytest.mark.parametrize("precision,tile_y,variant,tol", [("fp64", 0, 0, 1e-12), ("fp32", 0, 1, 1e-5),
                                                          ("fp32", 0, 2, 1e-5), ("fp32", 0, 3, 1e-5),
                                                          ("fp32", 4, 0, 1e-5)])
def test_full_size_single_step_128(built, oracle_mod, precision, tile_y, variant, tol):
    """128^3 with the benchmark's launch shape (fp32, automatic: the row-tiled
    cluster kernel) and the generic tile kernel: one step from an oracle state."""
    w = workloads.C2_THROUGHPUT
    box = (w.box,) * 3
    hist = w.gradient_history(3)
    o = oracle_mod.OracleLBM(box, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi))
    o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, hist[0])
    o.step(hist[0])
    f0 = inputs.perturbed_populations(o.populations(), 1e-4, seed=5)
    o.set_populations(f0)
    g = DropletLBM(box, w.R, w.visc, w.G, precision=precision, rho_hi=w.rho_hi, rho_lo=w.rho_lo, tile_y=tile_y,
                   row_variant=variant)
    g.set_populations(f0)
    g.set_gradient_table([0, 1, 2], hist)
    # the context's step counter is 0; the oracle steps with A(t=0) as well
    o.step(hist[0])
    g.step(1)
    assert rel_linf(g.populations(), o.populations()) <= tol


def test_moments_and_deformation_match_oracle(built, oracle_mod):
    box = (40, 36, 33)
    o, g = _pair(oracle_mod, box, 8.0, (1.0, 1.0), 3.5, "fp64")
    hist = inputs.ou_gradient_history(30, 10.0, 400.0, seed=9)
    o.init_droplet(8.0, 1.0, 1.0, workloads.RHO_LO, hist[0])
    o.run(30, np.arange(30), hist)
    g.set_populations(o.populations())
    from oracle.observables import deformation_from_moments

    m_ref = o.moments()
    m = g.moments()
    assert np.allclose(m, m_ref, rtol=1e-12, atol=1e-10)
    D_ref, axes_ref, lam_ref, c_ref = deformation_from_moments(m_ref)
    D, axes, lam, c = g.deformation()
    assert abs(D - D_ref) <= 1e-10 * abs(D_ref) + 1e-14
    assert np.allclose(lam, lam_ref, rtol=1e-10)
    assert np.allclose(c, c_ref, atol=1e-10)
    assert np.allclose(axes, axes_ref, atol=1e-8)


def test_checksums_and_periodic_conservation(built, oracle_mod):
    box = (20, 18, 16)
    o, g = _pair(oracle_mod, box, 4.0, (0.8, 1.4), 3.5, "fp64", periodic=True)
    o.init_droplet(4.0, 1.0, 1.0, workloads.RHO_LO, inputs.simple_shear(0.01))
    f0 = inputs.perturbed_populations(o.populations(), 1e-3, seed=4)
    g.set_populations(f0)
    m0, p0 = g.checksums()
    o.set_populations(f0)
    mo, po = o.checksums()
    assert np.allclose(m0, mo, rtol=1e-14) and np.allclose(p0, po, atol=1e-12)
    g.step(60)
    m1, p1 = g.checksums()
    assert np.all(np.abs(m1 - m0) <= 1e-12 * m0)
    assert np.all(np.abs(p1 - p0) <= 1e-12 * m0.sum())


def test_checkpoint_resume_is_bit_identical(built, tmp_path):
    w = workloads.C1_PARITY
    hist = inputs.ou_gradient_history(60, 20.0, 400.0, seed=8)
    mk = lambda: DropletLBM((24, 20, 22), 5.0, w.visc, w.G, precision="fp32", rho_lo=w.rho_lo)
    a = mk()
    a.set_gradient_table(np.arange(60), hist)
    a.step(60)
    ref = a.populations()
    b = mk()
    b.set_gradient_table(np.arange(60), hist)
    b.step(25)
    path = tmp_path / "ck.bin"
    b.save(path)
    c = mk()
    c.load(path)
    assert c.step_count() == 25
    c.step(35)
    assert np.array_equal(c.populations(), ref)
    # a corrupt file is rejected with LBM_EIO
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0xFF
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(LBMError) as e:
        mk().load(bad)
    assert e.value.code == -7


@pytest.mark.parametrize("box,precision", [((16, 16, 16), "fp32"), ((32, 16, 16), "fp32"), ((32, 16, 16), "fp16dev")])
def test_mach_guard_is_reported_not_faulted(built, box, precision):
    """The ghost kernel latches the Mach guard's error, before the generic
    kernel (16^3) and before the staged row kernel (32 x 16 x 16, float32
    and 16-bit deviation storage)."""
    w = workloads.C1_PARITY
    g = DropletLBM(box, 4.0, w.visc, w.G, precision=precision, rho_lo=w.rho_lo, mach_limit=0.5)
    g.set_gradient(inputs.simple_shear(0.2), 0)  # |u| >= 1.6 at the boundary
    g.step(2)
    with pytest.raises(LBMError) as e:
        g.sync()
    assert e.value.code == -5
    # the error stays latched
    with pytest.raises(LBMError):
        g.step(1)


def test_non_finite_input_rejected_on_host(built):
    w = workloads.C1_PARITY
    g = DropletLBM((8, 8, 8), 2.0, w.visc, w.G, precision="fp64", rho_lo=w.rho_lo)
    f = g.populations()
    f[0, 3, 2, 2, 2] = np.nan
    with pytest.raises(LBMError) as e:
        g.set_populations(f)
    assert e.value.code == -1
    with pytest.raises(LBMError):
        g.set_gradient(np.eye(3).reshape(9), 0)  # not traceless


def test_box_frame_short_run(built, oracle_mod):
    """The box-centred frame (ghost flow A x from the box centre), fp64."""
    box = (18, 16, 20)
    tau = (1.0, 1.1)
    o = oracle_mod.OracleLBM(box, tau, 3.5, (workloads.RHO_LO, 1.0), frame="box")
    g = DropletLBM(box, 4.0, ((tau[0] - 0.5) / 3, (tau[1] - 0.5) / 3), 3.5, precision="fp64", rho_hi=1.0,
                   rho_lo=workloads.RHO_LO, frame="box")
    A = inputs.simple_shear(0.01)
    o.init_droplet(4.0, 1.0, 1.0, workloads.RHO_LO, A)
    f0 = inputs.perturbed_populations(o.populations(), 1e-3, seed=6)
    o.set_populations(f0)
    g.set_populations(f0)
    g.set_gradient(A, 0)
    o.run(30, [0.0], [A])
    g.step(30)
    assert rel_linf(g.populations(), o.populations()) <= 1e-12


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("box", [(64, 24, 20), (128, 16, 9), (32, 40, 5), (256, 8, 6)])
def test_row_cluster_kernel_shapes(built, oracle_mod, box, variant):
    """The row-tiled cluster kernel (all variants) on other widths, cluster
    counts and short z extents (ragged last z chunk), fp32, 12 steps from a
    perturbed state."""
    tau = (1.0, 1.0)
    o, g = _pair(oracle_mod, box, 1.5, tau, 3.5, "fp32", z_chunk=2, row_variant=variant)
    hist = inputs.ou_gradient_history(12, 20.0, 600.0, seed=4)
    o.init_droplet(1.5, 1.0, 1.0, workloads.RHO_LO, hist[0])
    f0 = inputs.perturbed_populations(o.populations(), 1e-3, seed=8)
    o.set_populations(f0)
    g.set_populations(f0)
    g.set_gradient_table(np.arange(12), hist)
    o.run(12, np.arange(12), hist)
    g.step(12)
    assert rel_linf(g.populations(), o.populations()) <= 1e-5


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("box,z_chunk", [((128, 32, 40), 8), ((64, 16, 13), 5), ((32, 8, 6), 1)])
def test_row_variants_bit_identical(built, oracle_mod, precision, box, z_chunk):
    """Shared-memory staging with the populations carried in registers
    (variant 2) and loader and collider threads (variant 3) compute the same
    node updates as per-thread loads (variant 1) in the same order: with the
    same z chunks (hence the same march directions, centre-of-mass partials
    and frame origin) the stored states agree bit for bit after 25 steps of an
    OU-driven droplet, including chunks of one plane and ragged last chunks."""
    hist = inputs.ou_gradient_history(25, 20.0, 600.0, seed=11)
    R = min(box) / 4.0
    states = []
    for variant in (1, 2, 3):
        g = DropletLBM(box, R, (0.5 / 3, 0.5 / 3), 3.5, precision=precision, rho_hi=1.0, rho_lo=workloads.RHO_LO,
                       z_chunk=z_chunk, row_variant=variant)
        assert g.launch_shape()[1] == z_chunk
        g.set_gradient_table(np.arange(25), hist)
        g.step(25)
        states.append((g.populations(), g.deformation()[0]))
        g.close()
    for other in states[1:]:
        assert np.array_equal(states[0][0], other[0])
        assert states[0][1] == other[1]

