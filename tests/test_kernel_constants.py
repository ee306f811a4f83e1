"""Constants of the CUDA kernels checked against the mathematics they come from, on the
CPU: the coefficients of the inference GELU (Abramowitz & Stegun eq. 7.1.28, read out
of the kernel source) must give erfc within the published bound |error| <= 3e-7, and
the multiply-add chain must apply them in the order of the formula."""
import os
import re

import numpy as np
from scipy.special import erfc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2304_04781_gb300", "csrc", "aew_gemm.cuh")


def _fast_cdf_source() -> str:
    text = open(SRC).read()
    start = text.index("float normal_cdf_fast(float a)")
    return text[start:text.index("}", start)]


def _coefficients():
    """(c6, c5, c4, c3, c2, c1) in the nesting order of the kernel's Horner chain."""
    body = _fast_cdf_source()
    chain = body[body.index("float d ="):body.index(";", body.index("float d ="))]
    nums = [float(x.rstrip("f")) for x in re.findall(r"\d+\.\d+e-?\d+f|\d+\.\d+f", chain)]
    return nums


def test_gelu_coefficients_meet_the_published_bound():
    c6, c5, c4, c3, c2, c1 = _coefficients()
    z = np.linspace(0.0, 25.0, 2_500_001)
    d = 1.0 + z * (c1 + z * (c2 + z * (c3 + z * (c4 + z * (c5 + z * c6)))))
    err = np.abs(d ** -16.0 - erfc(z))
    assert err.max() <= 3e-7, err.max()
    # eq. 7.1.28's coefficients are positive and the polynomial starts at 1
    assert min(c1, c2, c3, c4, c5, c6) > 0.0
    body = _fast_cdf_source()
    assert "d = fmaf(d, z, 1.0f);" in body and body.count("d *= d;") == 4   # (.)^16
    assert "0.70710678118654752f" in body                                  # z = |a| / sqrt 2


def test_a_perturbed_coefficient_breaks_the_bound():
    """The check above can fail: the same chain with c1 off by 1% misses the bound."""
    c6, c5, c4, c3, c2, c1 = _coefficients()
    z = np.linspace(0.0, 25.0, 250_001)
    c1 *= 1.01
    d = 1.0 + z * (c1 + z * (c2 + z * (c3 + z * (c4 + z * (c5 + z * c6)))))
    assert np.abs(d ** -16.0 - erfc(z)).max() > 3e-7
