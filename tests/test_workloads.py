"""The seeded workload generators (CPU only): the suspensions every parity test
and the benchmark use are what their descriptions say -- capsule counts,
volume fractions, non-overlap with the 0.05a minimum gap, clearance from the
walls, outward triangle orientation, reproducibility from the seed."""
import math

import numpy as np
import pytest

from paper_1109_6587_gb300 import workloads as W


def _check_suspension(s, n_caps, nodes_per_cap):
    box = s.box
    assert s.x.shape == (n_caps * nodes_per_cap, 3)
    assert len(s.centres) == n_caps
    assert np.bincount(s.particle).tolist() == [nodes_per_cap] * n_caps
    # every node strictly inside the slit, with the 0.05a wall clearance
    assert s.x[:, 1].min() > box.y0 and s.x[:, 1].max() < box.y0 + box.W
    # centres at least 2a + 0.05a apart (minimum image in x and z)
    c = s.centres
    d = c[:, None, :] - c[None, :, :]
    d[..., 0] -= box.Lx * np.round(d[..., 0] / box.Lx)
    d[..., 2] -= box.Lz * np.round(d[..., 2] / box.Lz)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(n_caps) * 1e9
    assert r.min() >= (2.0 + 0.05) * s.radius - 1e-12
    # outward orientation: the signed volume of each capsule is positive
    x = s.x[s.tri]
    vol = np.einsum("ij,ij->i", x[:, 0], np.cross(x[:, 1], x[:, 2])) / 6.0
    per = np.bincount(s.particle[s.tri[:, 0]], weights=vol)
    assert (per > 0).all()


def test_benchmark_workload():
    s = W.capsules_100()
    _check_suspension(s, 100, 642)
    b = s.box
    assert (b.Lx, b.Lz, b.W, b.Nx, b.Ny, b.Nz) == (40.0, 40.0, 10.0, 128, 65, 128)
    s2 = W.capsules_100()
    assert np.array_equal(s.x, s2.x)                    # seeded


def test_volume_fraction_workloads():
    s = W.capsules_100_phi()
    _check_suspension(s, 382, 642)
    b = s.box
    phi = len(s.centres) * 4.0 / 3.0 * math.pi / (b.Lx * b.Lz * b.W)
    assert abs(phi - 0.1) < 2e-4
    # the larger one only by its count and fraction (placement is the same code)
    n = int(round(0.2 * 80.0 * 80.0 * 20.0 / (4.0 / 3.0 * math.pi)))
    assert n == 6112


@pytest.mark.parametrize("level,nodes", [(2, 162), (3, 642)])
def test_single_capsule_meshes(level, nodes):
    s = W.suspension(1, W.box_single_sphere(), level=level,
                     centres=np.array([[4.0, 0.0, 4.0]]))
    _check_suspension(s, 1, nodes)
    assert np.allclose(np.linalg.norm(s.x - s.centres[0], axis=1), 1.0)


def test_biconcave_workload():
    s = W.rbc_4000()
    _check_suspension(s, 4000, 642)
    # each cell is the Evans-Fung shape of radius 1: its volume is 1.56 R0^3
    x = s.x[s.tri]
    vol = np.einsum("ij,ij->i", x[:, 0], np.cross(x[:, 1], x[:, 2])) / 6.0
    per = np.bincount(s.particle[s.tri[:, 0]], weights=vol)
    assert np.allclose(per, per[0]) and abs(per[0] - 1.56) < 0.03
