"""Writes capsules100_phi_sampled.json and capsules1000_phi_sampled.json: the
oracle's FP64 single and double layer (nodal and element rule) at 100 sampled
nodes of the two workloads filled to the stated volume fractions --
workloads.capsules_100_phi() (382 capsules, 245,244 nodes, phi = 0.1, 40 x
[-5, 5] x 40, 128 x 65 x 128) and workloads.capsules_1000_phi() (6112
capsules, 3,923,904 nodes, phi = 0.2, 80 x [-10, 10] x 80, 256 x 97 x 256) --
for the full-size GPU parity tests.  Calls only oracle/ and the seeded
workload generators.  The second file takes about an hour on 8 cores.  Run
from the repository root:
    python tests/golden/make_phi.py [capsules100_phi | capsules1000_phi]
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                      # noqa: E402
from paper_1109_6587_gb300 import workloads as W    # noqa: E402

CASES = {"capsules100_phi": W.capsules_100_phi, "capsules1000_phi": W.capsules_1000_phi}


def sampled_layers(s, q, idx):
    box = s.box
    alpha = O.default_alpha(box)
    rcut = O.default_rcut(alpha)
    _, _, Ab, nb = O.geometry(s.x, s.tri)
    g = 8.0 * math.pi * Ab[:, None] * q
    xt = s.x[idx]
    # the global part once (velocity and stress), then each layer's local part
    ug, _, sg = O.global_fields(box, s.x, g, 1.0, alpha, rcut, want_stress=True)
    u_glob = O.interp(box, ug, xt)
    s_glob = np.einsum("nk,njk->nj", nb[idx], O.sym6_to_full(O.interp(box, sg, xt)))
    # nodal single layer as in O.point_forces: the self pair (r = 0) is left out
    # of the local sum and the free-space global self velocity is subtracted
    ul, _ = O.local_point(box, alpha, rcut, 1.0, s.x, g, xt, want_u=True, want_sig=False)
    w_nodal = ul + u_glob - (4.0 * alpha / math.sqrt(math.pi)) * g[idx] / (8.0 * math.pi)
    w_elem = O.local_elem(box, alpha, rcut, 0, s.x, s.tri, q, targets=idx) + u_glob
    v_elem = O.local_elem(box, alpha, rcut, 1, s.x, s.tri, q, nrm=nb, targets=idx) + s_glob
    return w_nodal, w_elem, v_elem


def main(names):
    for name in names:
        s = CASES[name]()
        n = s.x.shape[0]
        q = W.normal_forces(n, seed=8)
        idx = np.sort(np.random.default_rng(12).choice(n, 100, replace=False))
        w_nodal, w_elem, v_elem = sampled_layers(s, q, idx)
        out = {"source": "oracle/oracle.py via tests/golden/make_phi.py",
               "workload": f"workloads.{CASES[name].__name__}(), "
                           "q = workloads.normal_forces(n, seed=8)",
               "idx": idx.tolist(),
               "w_nodal": w_nodal.tolist(), "w_elem": w_elem.tolist(),
               "v_elem": v_elem.tolist()}
        with open(os.path.join(ROOT, "tests", "golden", f"{name}_sampled.json"), "w") as fh:
            json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
