"""Measurement probes that give the spreading's roofs (no counterpart in the
paper): float4 reductions into L2 (ggem_probe_l2_reduction) and FP32 atomic
adds into shared memory (ggem_probe_smem_reduction).  Checks that each runs,
times a launch and reports a rate within physical bounds, and that bad
arguments are refused before any device work."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def test_l2_reduction_probe(ggem):
    ms, rate = ggem.probe_l2_reduction(nvec=1 << 20, iters=64)
    assert ms > 0
    # 152 SMs cannot retire more than a few vector reductions per clock each
    assert 1e9 < rate < 152 * 8 * 2.2e9


def test_smem_reduction_probe(ggem):
    ms, rate = ggem.probe_smem_reduction(iters=512)
    assert ms > 0
    # at most 32 lanes per clock per SM
    assert 1e10 < rate < 152 * 32 * 2.2e9


def test_probe_argument_errors(ggem):
    with pytest.raises(ggem.GGEMError):
        ggem.probe_l2_reduction(nvec=33)
    with pytest.raises(ggem.GGEMError):
        ggem.probe_smem_reduction(iters=0)
