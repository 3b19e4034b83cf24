"""Run one layer operator on the 100-capsule workload, for profiling its kernels.

    python -m paper_1109_6587_gb300.profile_layer [precision] [layer]

precision: mixed (default), fp64 or fp64_emulated; layer: double (default) or
single.  Builds the element-rule plan, sets the mesh (64,200 nodes, 128 x 65 x
128 grid) and evaluates the layer twice for N(0,1) densities (seed 0), so a
profiler can skip the first evaluation's launches and capture the second's.
"""
import sys

import numpy as np
import torch

from paper_1109_6587_gb300 import ggem as G
from paper_1109_6587_gb300 import workloads as W


def main(argv):
    precision = argv[1] if len(argv) > 1 else "mixed"
    layer = argv[2] if len(argv) > 2 else "double"
    s = W.capsules_100()
    n = s.x.shape[0]
    P = G.Plan.for_box(s.box, precision=precision, quadrature="element", max_points=n,
                       max_tris=s.tri.shape[0])
    P.mesh_set(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.tri, device="cuda"))
    q = torch.as_tensor(np.random.default_rng(0).standard_normal((n, 3)), device="cuda")
    op = P.double_layer if layer == "double" else P.single_layer
    for _ in range(2):
        v = op(q)
    torch.cuda.synchronize()
    print("ok", float(v.abs().max()))


if __name__ == "__main__":
    main(sys.argv)
