"""Writes rbc4000_sampled.json: the oracle's FP64 single and double layer at
100 sampled nodes of the largest workload, 4000 biconcave capsules (2,568,000
nodes, 150 x [-15, 15] x 150 slit, 512 x 129 x 512 grid), for the full-size
GPU parity test.  Calls only oracle/ and the seeded workload generators.
Run from the repository root:
    python tests/golden/make_rbc4000.py
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


def main():
    s = W.rbc_4000()
    n = s.x.shape[0]
    q = W.normal_forces(n, seed=8)
    idx = np.sort(np.random.default_rng(12).choice(n, 100, replace=False))
    box = s.box
    alpha = O.default_alpha(box)
    rcut = O.default_rcut(alpha)
    _, _, Ab, nb = O.geometry(s.x, s.tri)
    g = 8.0 * math.pi * Ab[:, None] * q
    xt = s.x[idx]
    # global part once (velocity and stress), then each layer's local part
    ug, _, sg = O.global_fields(box, s.x, g, 1.0, alpha, rcut, want_stress=True)
    u_glob = O.interp(box, ug, xt)
    s_glob = np.einsum("nk,njk->nj", nb[idx], O.sym6_to_full(O.interp(box, sg, xt)))
    # nodal single layer: point forces at the nodes themselves, combined as in
    # O.point_forces (the self pair has r = 0 and is left out of the local sum;
    # the free-space global self velocity is subtracted)
    ul, _ = O.local_point(box, alpha, rcut, 1.0, s.x, g, xt, want_u=True, want_sig=False)
    w_nodal = ul + u_glob - (4.0 * alpha / math.sqrt(math.pi)) * g[idx] / (8.0 * math.pi)
    w_elem = O.local_elem(box, alpha, rcut, 0, s.x, s.tri, q, targets=idx) + u_glob
    v_elem = O.local_elem(box, alpha, rcut, 1, s.x, s.tri, q, nrm=nb, targets=idx) + s_glob
    out = {"source": "oracle/oracle.py via tests/golden/make_rbc4000.py",
           "workload": "workloads.rbc_4000(), q = workloads.normal_forces(n, seed=8)",
           "idx": idx.tolist(),
           "w_nodal": w_nodal.tolist(), "w_elem": w_elem.tolist(), "v_elem": v_elem.tolist()}
    with open(os.path.join(ROOT, "tests", "golden", "rbc4000_sampled.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
