"""Write tests/golden/shan_chen_G3.5_tau1.json from the FP64 oracle alone.

Run from the repository root:  python tests/golden/make_golden.py

Measures, for the Shan-Chen coupling G = 3.5 at tau = 1 (Sec. 2, Eq. 7):
* the discrete flat-interface coexistence densities (a periodic 1D slab
  relaxed for 20000 steps); the minority value is used as the ghost density
  rho_b of the droplet component, so that the open boundary (Sec. 3) neither
  feeds nor drains the droplet at rest;
* the surface tension sigma from Laplace's law dp = 2 sigma/R for spherical
  droplets (R = 6, 8 in a periodic 28^3 box, 3000 steps), with the bulk
  pressure p = c_s^2 (rho_A + rho_B) + G c_s^2 rho_A rho_B.
sigma sets the shear rate of a given capillary number (Eq. 3).
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.observables import bulk_pressure, coexistence_rho_lo  # noqa: E402

G, TAU = 3.5, 1.0


def flat_coexistence():
    L = 64
    lo0 = coexistence_rho_lo(G)
    o = oracle.OracleLBM((L, 1, 1), (TAU, TAU), G, (lo0, 1.0), periodic=True)
    o.init_droplet(16.0, 1.0, 1.0, lo0)
    o.run(20000)
    ra, rb, _ = o.fields()
    return float(ra.max()), float(ra.min())


def sphere_sigma(L, R, steps=3000):
    lo0 = coexistence_rho_lo(G)
    o = oracle.OracleLBM((L, L, L), (TAU, TAU), G, (lo0, 1.0), periodic=True)
    o.init_droplet(R, 1.0, 1.0, lo0)
    o.run(steps)
    ra, rb, _ = o.fields()
    c = (L // 2, L // 2, L // 2)
    dp = bulk_pressure(ra[c], rb[c], G) - bulk_pressure(ra[0, 0, 0], rb[0, 0, 0], G)
    vol = np.sum((ra - ra[0, 0, 0]) / (ra[c] - ra[0, 0, 0]))
    Reff = (3 * vol / (4 * np.pi)) ** (1 / 3)
    return float(dp * Reff / 2), float(Reff)


def main():
    oracle.set_threads(os.cpu_count() or 1)
    hi, lo = flat_coexistence()
    sig = [sphere_sigma(28, R) for R in (6.0, 8.0)]
    out = {
        "G": G,
        "tau": TAU,
        "flat_rho_hi": round(hi, 6),
        "flat_rho_lo": round(lo, 6),
        "sigma": round(float(np.mean([s for s, _ in sig])), 4),
        "sigma_by_radius": [{"R_eff": round(r, 3), "sigma": round(s, 5)} for s, r in sig],
        "written_by": "python tests/golden/make_golden.py (FP64 oracle only)",
    }
    with open(os.path.join(HERE, "shan_chen_G3.5_tau1.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
