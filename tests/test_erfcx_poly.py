"""The pair kernels form erfc(x) = exp(-x^2) erfcx(x) with the approximations
of ggem_erfcx.cuh on 0 <= x <= 4 (alpha r inside the cutoff).  FP32:
erfcx(x) ~ t Q(t), t = 1/(1 + P x), Q of degree 6 in t.  Its coefficients, read
from the generated header, must approximate scipy's erfcx to 2e-7 relative in
FP64 (about the rounding of its own FP32 evaluation) and to 5e-7 (a few FP32
ulps, like CUDA's erfcf) when t and the Horner scheme are evaluated in FP32.
FP64: 8 pieces of degree 12."""
import pathlib
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

HDR = pathlib.Path(__file__).resolve().parents[1] / "paper_1109_6587_gb300" / "csrc" / "ggem_erfcx.cuh"


def _coefficients():
    txt = HDR.read_text()
    first = re.search(r"float q = ([-+0-9.eE]+)f;", txt).group(1)
    rest = re.findall(r"q = fmaf\(q, t, ([-+0-9.eE]+)f\);", txt)
    return [float(first)] + [float(v) for v in rest]    # highest degree first


def _p():
    return float(re.search(r"#define GGEM_ERFCX_P ([0-9.]+)f", HDR.read_text()).group(1))


def _table64():
    txt = HDR.read_text()
    body = re.search(r"kErfcxTab64\[\d+\] = \{(.*?)\};", txt, re.S).group(1)
    vals = [float(v) for v in re.findall(r"[-+]?\d\.\d+e[-+]\d+", body)]
    return np.array(vals).reshape(13, 8)          # [power][interval]

def test_polynomial_error():
    c = _coefficients()
    assert len(c) == 7
    p = _p()
    x = np.linspace(0.0, 4.0, 100001)
    ref = special.erfcx(x)
    t = 1.0 / (1.0 + p * x)
    q = np.full_like(t, c[0])
    for a in c[1:]:
        q = q * t + a
    assert np.abs(q * t / ref - 1).max() < 2e-7
    x32 = x.astype(np.float32)
    t32 = (np.float32(1) / (np.float32(p) * x32 + np.float32(1))).astype(np.float32)
    q32 = np.full_like(t32, np.float32(c[0]))
    for a in c[1:]:
        q32 = (q32 * t32 + np.float32(a)).astype(np.float32)
    q32 = (q32 * t32).astype(np.float32)
    assert np.abs(q32.astype(np.float64) / ref - 1).max() < 5e-7


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
    first = re.search(r"f2 q = f2_splat\(([-+0-9.eE]+)f\);", txt).group(1)
    rest = re.findall(r"q = fma2\(q, t, f2_splat\(([-+0-9.eE]+)f\)\);", txt)
    assert [float(first)] + [float(v) for v in rest] == _coefficients()
