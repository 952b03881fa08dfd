"""The allocation-free moments entry point agrees with the context-based one.

lbm_moments_static serves callers that cannot allocate device memory when
they need the droplet's shape (for example code recording into a CUDA graph).
It keeps its scratch in a fixed device array shared by all calls; this test
calls it twice in a row through the C ABI, on float64 and float32 population
arrays the caller holds on the device, and compares both results with
lbm_moments / lbm_deformation of the same state.  This file is collected
last so that a failure here cannot hide failures elsewhere.
"""

import numpy as np
import pytest

from paper_2112_09972_gb300 import inputs, workloads
from paper_2112_09972_gb300.lbm import DropletLBM, lbm_moments_static

pytestmark = pytest.mark.gpu


def test_static_moments_match_context_moments():
    import torch

    from paper_2112_09972_gb300 import build

    build.build()
    w = workloads.C1_PARITY
    box = (40, 34, 30)
    g = DropletLBM(box, 7.0, w.visc, w.G, precision="fp64", rho_lo=w.rho_lo)
    hist = inputs.ou_gradient_history(30, 20.0, 150.0, seed=3)
    g.set_gradient_table(np.arange(30), hist)
    g.step(30)
    ref_m = g.moments()
    ref_D, ref_axes, ref_lam, ref_c = g.deformation()
    f = g.populations()
    stream = torch.cuda.current_stream()
    for dtype, prec, rtol in ((torch.float64, "fp64", 1e-12), (torch.float32, "fp32", 1e-6)):
        f_dev = torch.from_numpy(f).to(device="cuda", dtype=dtype).contiguous()
        for call in range(2):  # two calls in a row share the scratch array
            out = torch.full((26,), float("nan"), dtype=torch.float64, device="cuda")
            lbm_moments_static(f_dev.data_ptr(), prec, box, out.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            r = out.cpu().numpy()
            assert np.allclose(r[:10], ref_m, rtol=rtol, atol=rtol * 1e-3 * abs(ref_m[0])), (prec, call)
            assert abs(r[10] - ref_D) <= 10 * rtol * abs(ref_D) + 1e-12, (prec, call)
            assert np.allclose(r[20:23], ref_lam, rtol=10 * rtol), (prec, call)
            assert np.allclose(r[23:26], ref_c, atol=10 * rtol * 10), (prec, call)
            axes = r[11:20].reshape(3, 3)
            for k in range(3):
                gap = min(abs(ref_lam[k] - ref_lam[j]) for j in range(3) if j != k) / abs(ref_lam[0])
                if gap > 1e-3:  # the axis is well defined
                    assert abs(abs(axes[:, k] @ ref_axes[:, k]) - 1) < 1e-6, (prec, call)
    g.close()


def test_static_moments_rejects_invalid_sizes():
    import torch

    f_dev = torch.zeros(38, dtype=torch.float64, device="cuda")
    out = torch.zeros(26, dtype=torch.float64, device="cuda")
    from paper_2112_09972_gb300.lbm import LBMError

    with pytest.raises(LBMError):
        lbm_moments_static(f_dev.data_ptr(), "fp64", (0, 1, 1), out.data_ptr())
    with pytest.raises(LBMError):
        lbm_moments_static(f_dev.data_ptr(), "fp64", (2048, 2048, 2048), out.data_ptr())
