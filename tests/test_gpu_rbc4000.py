"""Full-size parity on the largest workload: 4000 biconcave capsules x 642
nodes (2,568,000 nodes, Evans-Fung profile, random orientations; 150 x
[-15, 15] x 150 slit, 512 x 129 x 512 grid).  The single and double layer at
every node on the GPU, compared at 100 sampled nodes with the oracle's FP64
values stored by tests/golden/make_rbc4000.py.  Tolerances as everywhere:
1e-10 (FP64 and FP64-emulated), 1e-5 (mixed), max |gpu - oracle| /
max |oracle| over the sampled outputs."""
import json
import pathlib

import numpy as np
import pytest
from _parity import assert_close

from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp64_emulated": 1e-10, "mixed": 1e-5}
GOLD = pathlib.Path(__file__).resolve().parent / "golden" / "rbc4000_sampled.json"


@pytest.fixture(scope="module")
def case():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    ref = json.loads(GOLD.read_text())
    s = W.rbc_4000()
    q = W.normal_forces(s.x.shape[0], seed=8)
    return G, s, q, ref


def _rel(a, b):
    b = np.asarray(b)
    return np.abs(np.asarray(a) - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec,quad", [("mixed", "nodal"), ("mixed", "element"),
                                       ("fp64_emulated", "element"), ("fp64", "nodal"),
                                       ("fp64", "element")])
def test_rbc4000_layers(case, prec, quad):
    G, s, q, ref = case
    idx = np.asarray(ref["idx"])
    P = G.Plan.for_box(s.box, precision=prec, quadrature=quad, max_points=s.x.shape[0],
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
