"""FP64 CPU oracle of the paper's method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call or run anything in this package.  It shares no
code with the CUDA library in ``paper_2112_09972_gb300`` and imports nothing
from it.

* ``lbm``          -- the two-component Shan-Chen LBM step (Sec. 2, Eqs. 6-10),
                      ghost-node exact-flow boundary (Sec. 3, Eq. 14).
* ``observables``  -- D from the inertia tensor (Eq. 4), E^(0) (Eq. 16),
                      bulk pressure and flat-interface coexistence (Eq. 7).
* ``mm``           -- the Maffettone-Minale model (Eqs. 1, 2, 5).

Parity pins live in ``tests/test_oracle_*.py``.  Functions whose result the
paper does not fix independently are listed there; none is unpinned.
"""

from .lbm import OracleLBM, gradient_at, lattice, equilibrium, set_threads  # noqa: F401
from . import observables, mm  # noqa: F401
