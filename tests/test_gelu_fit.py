"""The normal-CDF fit behind the surrogate's GELU epilogues: the fitting
script beside the kernels reproduces the coefficients the kernels hold and
the error bounds their documentation states (|Phi_a - Phi| < 6.8e-6,
|z| |Phi_a - Phi| < 3.1e-6 over the fit's grid).  CPU only."""
from __future__ import annotations

import os
import re
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2406_08496_gb300", "csrc")


def _kernel_coefficients():
    src = open(os.path.join(CSRC, "mlp.cu")).read()
    body = src[src.index("__device__ __forceinline__ float norm_cdf(float z)"):]
    body = body[:body.index("}")]
    return [float(x) for x in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]


def test_fit_reproduces_the_kernel_constants_and_bounds():
    sys.path.insert(0, CSRC)
    try:
        import fit_normal_cdf as F
    finally:
        sys.path.pop(0)
    c, err_gelu, err_phi = F.fit()
    assert err_gelu < 3.1e-6 and err_phi < 6.8e-6, (err_gelu, err_phi)
    k = _kernel_coefficients()
    # Horner order in the kernel: c4, c3, c2, c1, c0
    assert len(k) == 5
    assert np.array_equal(np.float32(k[::-1]), c), (k, c)
