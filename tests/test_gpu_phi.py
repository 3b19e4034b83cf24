"""Full-size parity on the workloads filled to the stated volume fractions:
the 100-capsule slit and grid at phi = 0.1 (382 capsules, 245,244 nodes) and
the 1000-capsule slit and grid at phi = 0.2 (6112 capsules, 3,923,904
nodes).  The single and double layer at every node on the GPU, compared at
100 sampled nodes with the oracle's FP64 values stored by
tests/golden/make_phi.py.  Tolerances as everywhere: 1e-10 (FP64 and
FP64-emulated), 1e-5 (mixed), max |gpu - oracle| / max |oracle| over the
sampled outputs.  (The native-FP64 element rule on the larger workload, about
a minute per layer at GB300's FP64 rate, is covered by the FP64-emulated
plan at the FP64 bar.)"""
import json
import pathlib

import numpy as np
import pytest
from _parity import assert_close

from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp64_emulated": 1e-10, "mixed": 1e-5}
GOLD = pathlib.Path(__file__).resolve().parent / "golden"
CASES = {"capsules100_phi": W.capsules_100_phi, "capsules1000_phi": W.capsules_1000_phi}
RUNS = [("capsules100_phi", "mixed", "nodal"), ("capsules100_phi", "mixed", "element"),
        ("capsules100_phi", "fp64_emulated", "element"), ("capsules100_phi", "fp64", "nodal"),
        ("capsules100_phi", "fp64", "element"),
        ("capsules1000_phi", "mixed", "nodal"), ("capsules1000_phi", "mixed", "element"),
        ("capsules1000_phi", "fp64_emulated", "element"), ("capsules1000_phi", "fp64", "nodal")]


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


_cache = {}


def _case(name):
    if name not in _cache:
        _cache.clear()                          # one workload in host memory at a time
        s = CASES[name]()
        q = W.normal_forces(s.x.shape[0], seed=8)
        ref = json.loads((GOLD / f"{name}_sampled.json").read_text())
        _cache[name] = (s, q, ref)
    return _cache[name]


def _rel(a, b):
    b = np.asarray(b)
    return np.abs(np.asarray(a) - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name,prec,quad", RUNS)
def test_phi_layers(ggem, name, prec, quad):
    s, q, ref = _case(name)
    idx = np.asarray(ref["idx"])
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature=quad, max_points=s.x.shape[0],
                          max_tris=s.tri.shape[0])
    dev = torch.device("cuda")
    P.mesh_set(torch.as_tensor(s.x, device=dev), torch.as_tensor(s.tri, device=dev))
    qd = torch.as_tensor(q, device=dev)
    w = P.single_layer(qd).cpu().numpy()[idx]
    if quad == "nodal":
        assert_close(w, ref["w_nodal"], TOL[prec])
    else:
        assert_close(w, ref["w_elem"], TOL[prec])
        v = P.double_layer(qd).cpu().numpy()[idx]
        assert_close(v, ref["v_elem"], TOL[prec])
    P.check()
    P.close()
