"""Failure detection on the GPU without a fault: a bounded wait made to expire.

The tensor-core Chebyshev transform waits on an mbarrier for its MMAs with an
iteration limit.  ggem_inject_tc_wait_expiry makes the next launch issue no
MMA for its first tile and poll only 1,000 times, so the wait runs out with
nothing in flight.  The plan must report it (ggem_check: GGEM_ERR_CUDA) and
the CUDA context must stay usable: a fresh plan then evaluates the single
layer to the mixed-precision parity with the oracle and reports no failure.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _case(ggem):
    s = W.single_sphere(radius=0.97)
    q = W.normal_forces(s.x.shape[0], seed=3)
    P = ggem.Plan.for_box(s.box, precision="mixed", max_points=1000, max_tris=1000)
    P.mesh_set(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.tri, device="cuda"))
    return s, q, P


def test_expired_tensor_core_wait_is_reported_and_the_context_survives(ggem):
    s, q, P = _case(ggem)
    qd = torch.as_tensor(q, device="cuda")
    assert ggem.lib().ggem_inject_tc_wait_expiry(1000) == 0
    P.single_layer(qd)                         # the forward transform gives up waiting
    with pytest.raises(ggem.GGEMError) as e:
        P.check()
    assert e.value.status == 3                 # GGEM_ERR_CUDA
    P.close()
    # a fresh plan on the same device: correct results, no failure recorded
    _, _, P2 = _case(ggem)
    w = P2.single_layer(qd).cpu().numpy()
    ref = O.single_layer(s, q, quadrature="nodal")
    assert np.abs(w - ref).max() < 1e-5 * np.abs(ref).max()
    P2.check()
    # the injection applies to one launch only
    w2 = P2.single_layer(qd).cpu().numpy()
    assert np.abs(w2 - ref).max() < 1e-5 * np.abs(ref).max()
    P2.check()
    assert ggem.lib().ggem_inject_tc_wait_expiry(0) == 1          # out of range
    P2.close()
