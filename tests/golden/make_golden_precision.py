"""Write tests/golden/precision_downscale64.json from the FP64 oracle alone.

Run from the repository root:  python tests/golden/make_golden_precision.py

The precision case (256^3, R = 32, 16-bit deviation storage) is compared
with the FP64 oracle on its 64^3, R = 8 downscale: the same OU gradient
history (seed and Eq. 15 velocity scale u_LBM), rescaled to the small box.
This script runs that downscale on the oracle for STEPS steps from the
equilibrium tanh droplet and stores the droplet's deformation D, its axes,
eigenvalues and centre (Sec. 2, Eq. 4), the component masses, and the
density and velocity at a fixed seeded sample of nodes, so that the
benchmark can state each storage form's error against the FP64 oracle
without running the oracle itself.
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.observables import deformation_from_moments  # noqa: E402
from paper_2112_09972_gb300 import workloads  # noqa: E402

STEPS = 400
NSAMPLE = 256


def sample_nodes(box, n, seed=12350):
    """Seeded sample of node indices (z, y, x) of a box."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0]))
    return np.stack([rng.integers(0, box[2], n), rng.integers(0, box[1], n), rng.integers(0, box[0], n)], axis=1)


def main():
    oracle.set_threads(os.cpu_count() or 1)
    w = workloads.C4_DOWNSCALED
    box = (w.box,) * 3
    hist = w.gradient_history(STEPS + 1)
    o = oracle.OracleLBM(box, (w.tau, w.tau), w.G, (w.rho_lo, w.rho_hi))
    o.init_droplet(w.R, w.xi, w.rho_hi, w.rho_lo, hist[0])
    o.run(STEPS, np.arange(STEPS + 1), hist)
    D, axes, lam, centre = deformation_from_moments(o.moments())
    ra, rb, u = o.fields()
    idx = sample_nodes(box, NSAMPLE)
    z, y, x = idx[:, 0], idx[:, 1], idx[:, 2]
    out = {
        "workload": w.name,
        "steps": STEPS,
        "D": float(D),
        "axes": np.asarray(axes).tolist(),
        "lambda": np.asarray(lam).tolist(),
        "centre": np.asarray(centre).tolist(),
        "mass": o.checksums()[0].tolist(),
        "sample_nodes_zyx": idx.tolist(),
        "rho_a": ra[z, y, x].tolist(),
        "rho_b": rb[z, y, x].tolist(),
        "u": u[z, y, x].tolist(),
        "rho_a_max": float(ra.max()),
        "u_max": float(np.abs(u).max()),
        "written_by": "python tests/golden/make_golden_precision.py (FP64 oracle only)",
    }
    with open(os.path.join(HERE, "precision_downscale64.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps({k: out[k] for k in ("workload", "steps", "D", "lambda", "mass")}, indent=1))


if __name__ == "__main__":
    main()
