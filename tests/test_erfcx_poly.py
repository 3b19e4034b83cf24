"""The pair kernels form erfc(x) = exp(-x^2) erfcx(x) with the polynomials of
ggem_erfcx.cuh on 0 <= x <= 4 (alpha r inside the cutoff): degree 14 (FP32),
8 pieces of degree 12 (FP64).  FP32:
Its coefficients, read from the generated header, must approximate scipy's
erfcx to 2e-7 relative in FP64 (the approximation error is kept near the
rounding error of the polynomial's own FP32 evaluation, ~2e-7, so neither
dominates) and to 4e-7 (a few FP32 ulps, like CUDA's erfcf) when evaluated in
FP32 by the same Horner scheme."""
import pathlib
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

HDR = pathlib.Path(__file__).resolve().parents[1] / "paper_1109_6587_gb300" / "csrc" / "ggem_erfcx.cuh"


def _coefficients():
    txt = HDR.read_text()
    first = re.search(r"float p = ([-+0-9.eE]+)f;", txt).group(1)
    rest = re.findall(r"p = fmaf\(p, u, ([-+0-9.eE]+)f\);", txt)
    return [float(first)] + [float(v) for v in rest]    # highest degree first


def _table64():
    txt = HDR.read_text()
    body = re.search(r"kErfcxTab64\[\d+\] = \{(.*?)\};", txt, re.S).group(1)
    vals = [float(v) for v in re.findall(r"[-+]?\d\.\d+e[-+]\d+", body)]
    return np.array(vals).reshape(13, 8)          # [power][interval]

def test_polynomial_error():
    c = _coefficients()
    assert len(c) == 15
    x = np.linspace(0.0, 4.0, 100001)
    ref = special.erfcx(x)
    u = x / 2 - 1
    p = np.full_like(u, c[0])
    for a in c[1:]:
        p = p * u + a
    assert np.abs(p / ref - 1).max() < 2e-7
    x32 = x.astype(np.float32)
    u32 = (x32 * np.float32(0.5) - np.float32(1)).astype(np.float32)
    p32 = np.full_like(u32, np.float32(c[0]))
    for a in c[1:]:
        p32 = (p32 * u32 + np.float32(a)).astype(np.float32)
    assert np.abs(p32.astype(np.float64) / ref - 1).max() < 4e-7


def test_polynomial_error_fp64():
    """The FP64 kernels' 8 pieces of degree 12 ([i/2, (i+1)/2], u = 4x - 2i - 1)
    against mpmath at 40 digits: 3e-15 relative (FP64 parity of the pair sums
    is 1e-10)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    tab = _table64()
    x = np.linspace(0.0, 4.0, 801)
    ref = np.array([float(mp.exp(mp.mpf(v) ** 2) * mp.erfc(mp.mpf(v))) for v in x])
    i = np.minimum((x * 2.0).astype(int), 7)
    u = 4.0 * x - (2.0 * i + 1.0)
    p = tab[12, i]
    for j in range(11, -1, -1):
        p = p * u + tab[j, i]
    assert np.abs(p / ref - 1).max() < 3e-15


def test_paired_polynomial_has_the_same_coefficients():
    # the paired-lane copy used by the FP32 element-rule kernel
    txt = HDR.read_text()
    first = re.search(r"f2 p = f2_splat\(([-+0-9.eE]+)f\);", txt).group(1)
    rest = re.findall(r"p = fma2\(p, u, f2_splat\(([-+0-9.eE]+)f\)\);", txt)
    assert [float(first)] + [float(v) for v in rest] == _coefficients()
