"""ggem_local_velocity_noalloc against ggem_local_sum, through the C ABI.

The allocation-free entry point exists for callers that cannot call
cudaMalloc -- code recording a CUDA graph under stream capture, programs whose
device memory is owned by another allocator or a fixed budget, loops that must
not pay cudaFree's device-wide synchronisation -- and so cannot create a plan.
It must give the same local velocity as the plan-based ggem_local_sum.  Two
calls are made in a row with different inputs, the second with fewer sources,
because both share one scratch array that keeps the previous call's contents.
"""
import ctypes

import numpy as np
import pytest

from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_plan_local_sum_on_two_calls():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem

    L = ggem.lib()
    fn = L.ggem_local_velocity_noalloc
    fn.argtypes = [ctypes.POINTER(ggem.ggem_params), ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int

    s = W.capsules_100()
    box = s.box
    n = s.x.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    n_chunked = 70_000          # more free targets than one chunk of the scratch array
    plan = ggem.Plan.for_box(box, precision="fp64", max_points=max(n, n_chunked), stream=stream)
    prm = ggem.ggem_params(box.Lx, box.Lz, box.W, box.y0, box.Nx, box.Ny, box.Nz,
                           0.0, 0.0, 1.0, ggem.GGEM_FP64, ggem.GGEM_NODAL, 0, 0)
    rng = np.random.default_rng(21)
    for call, ns in enumerate((n, 40_000)):
        xs = _dev(s.x[:ns])
        g = _dev(W.normal_forces(ns, seed=30 + call))
        xt = _dev(s.x[rng.choice(n, 500, replace=False)] + rng.normal(scale=0.1, size=(500, 3)))
        ref, _ = plan.local_sum(xs, g, xt)
        u = torch.full((500, 3), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(ctypes.byref(prm), ctypes.c_void_p(stream), ns, _p(xs), _p(g), 500, _p(xt), 0,
                _p(u))
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        err = float((u - ref).abs().max() / ref.abs().max())
        assert err < TOL_FP64, f"call {call}: rel err {err}"
        # targets = sources
        refs, _ = plan.local_sum(xs, g)
        us = torch.full((ns, 3), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(ctypes.byref(prm), ctypes.c_void_p(stream), ns, _p(xs), _p(g), 0, None, 1,
                _p(us))
        assert st == 0
        torch.cuda.synchronize()
        assert float((us - refs).abs().max() / refs.abs().max()) < TOL_FP64

    # free targets beyond one chunk (GGEM_NOALLOC_MAX_POINTS): located and summed
    # chunk by chunk, same result
    ns = 30_000
    xs = _dev(s.x[:ns])
    g = _dev(W.normal_forces(ns, seed=40))
    pick = rng.choice(n, n_chunked, replace=True)
    xt = _dev(s.x[pick] + rng.normal(scale=0.2, size=(n_chunked, 3)) * [1.0, 0.0, 1.0])
    ref, _ = plan.local_sum(xs, g, xt)
    u = torch.full((n_chunked, 3), float("nan"), dtype=torch.float64, device="cuda")
    st = fn(ctypes.byref(prm), ctypes.c_void_p(stream), ns, _p(xs), _p(g), n_chunked, _p(xt), 0,
            _p(u))
    assert st == 0, f"chunked targets: status {st}"
    torch.cuda.synchronize()
    err = float((u - ref).abs().max() / ref.abs().max())
    assert err < TOL_FP64, f"chunked targets: rel err {err}"

    # beyond the stated maximum: a clear capacity error, no device work
    big = ggem.ggem_params(box.Lx, box.Lz, box.W, box.y0, box.Nx, box.Ny, box.Nz,
                           0.0, 0.0, 1.0, 0, 0, 0, 0)
    u = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    st = fn(ctypes.byref(big), ctypes.c_void_p(stream), 70_000, _p(u), _p(u), 1, _p(u), 0, _p(u))
    assert st == 2
    # a cell grid larger than GGEM_NOALLOC_MAX_CELLS (an 800 x 800 slit with
    # cells of r_cut = 3.1: 256 x 3 x 256 cells): capacity error, no device work
    wide = ggem.ggem_params(800.0, 800.0, box.W, box.y0, 2048, box.Ny, 2048,
                            0.0, 0.0, 1.0, 0, 0, 0, 0)
    st = fn(ctypes.byref(wide), ctypes.c_void_p(stream), 10, _p(u), _p(u), 1, _p(u), 0, _p(u))
    assert st == 2
