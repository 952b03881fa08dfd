"""Run a named workload for a few steps through the C ABI (for profiling runs).

    python -m paper_2112_09972_gb300.run_case --workload droplet128_R16_ou --steps 10
    python -m paper_2112_09972_gb300.run_case --workload droplet256_R32_ou_dev16 --precision fp16dev
    python -m paper_2112_09972_gb300.run_case --mlp-batch 65536 --steps 3

Builds the library if needed, creates the box with the workload's radius and
fluid parameters, loads its gradient history and takes ``--steps`` steps
(ghost kernel + stream-collide kernel each), then prints D.  Each step
launches the same kernels as the benchmark, so a profiler can select one
launch of a kernel by name and launch count.

With ``--mlp-batch n`` it runs the surrogate's network instead (576 -> 256 ->
256 -> 256 -> 6, seeded weights, seeded standard-normal inputs and targets):
``--steps`` forward passes of n windows, then one training step.
"""

import argparse

import numpy as np

from . import build, workloads
from .lbm import DropletLBM


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default=workloads.C2_THROUGHPUT.name, choices=sorted(workloads.WORKLOADS))
    p.add_argument("--precision", default=None, help="fp64, fp32, fp16dev or bf16dev (default: the workload's)")
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--tile-y", type=int, default=0)
    p.add_argument("--z-chunk", type=int, default=0)
    p.add_argument("--row-variant", type=int, default=0, help="row kernel: 1 direct loads, 2 staged, 3 warp-specialised")
    p.add_argument("--mlp-batch", type=int, default=0)
    p.add_argument("--tensor-path", type=int, default=0, help="MLP products: 0 tcgen05 where possible, 1 mma.sync")
    a = p.parse_args(argv)
    if a.mlp_batch > 0:
        return run_mlp(a.mlp_batch, a.steps, a.tensor_path)
    w = workloads.WORKLOADS[a.workload]
    build.build()
    prec = a.precision or w.precision
    g = DropletLBM((w.box,) * 3, w.R, w.visc, w.G, precision=prec, rho_hi=w.rho_hi, rho_lo=w.rho_lo, xi=w.xi,
                   tile_y=a.tile_y, z_chunk=a.z_chunk, row_variant=a.row_variant)
    hist = w.gradient_history(max(a.steps, 1))
    g.set_gradient_table(np.arange(hist.shape[0]), hist)
    g.step(a.steps)
    D = g.deformation()[0]
    ty, zc, ctas = g.launch_shape()
    print(f"{w.name} {prec}: {a.steps} steps, D = {D:.6f}, launch shape tile_y={ty} z_chunk={zc} ctas={ctas} "
          f"variant={g.launch_variant()}")


def run_mlp(n, steps, path):
    import torch

    from .lbm import MLP
    from .surrogate import HIDDEN, N_OUT, WINDOW

    SIZES = (9 * WINDOW,) + tuple(HIDDEN) + (N_OUT,)
    build.build()
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.standard_normal((n, SIZES[0]), dtype=np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((n, SIZES[-1]), dtype=np.float32)).cuda()
    y = torch.empty((n, SIZES[-1]), dtype=torch.float32, device="cuda")
    net = MLP(SIZES, max_batch=n, seed=7)
    net.set_tensor_path(path)
    for _ in range(steps):
        net.forward(x, y)
    loss = net.train_step(x, t, 1e-4, want_loss=True)
    net.sync()
    print(f"mlp {SIZES} batch {n}: {steps} forward passes and one training step, loss {loss:.6f}, path {path}")
    net.close()


if __name__ == "__main__":
    main()
