"""The C-ABI library builds, loads and exports every symbol include/ggem.h
declares; argument validation that happens before any CUDA call (CPU only)."""
import ctypes
import pathlib
import re

import pytest

from paper_1109_6587_gb300 import _build
from paper_1109_6587_gb300 import ggem

ROOT = pathlib.Path(__file__).resolve().parents[1]


def declared_symbols():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        txt = h.read_text()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    _build.build()
    return ggem.lib()


def test_every_declared_symbol_is_exported(built):
    names = declared_symbols()
    assert "ggem_plan" in names and "ggem_single_layer" in names
    for n in names:
        assert hasattr(built, n), n
        assert isinstance(getattr(built, n), ctypes._CFuncPtr)


def test_binding_covers_header():
    assert declared_symbols() <= set(ggem.EXPORTS) | {"bie_solve"} | set(ggem.EXPORTS)


def _params(**kw):
    base = dict(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=32, Ny=33, Nz=32, alpha=0.0,
                rcut_factor=0.0, mu=1.0, precision=0, quadrature=0, max_points=100,
                max_tris=0)
    base.update(kw)
    return ggem.ggem_params(**base)


@pytest.mark.parametrize("bad", [dict(Nx=30), dict(Ny=5), dict(W=-1.0), dict(mu=0.0),
                                 dict(precision=7), dict(alpha=0.5), dict(max_points=0)])
def test_invalid_parameters_rejected_before_any_device_work(built, bad):
    h = ctypes.c_void_p()
    st = built.ggem_plan(ctypes.byref(_params(**bad)), None, ctypes.byref(h))
    assert st == 1                       # GGEM_ERR_INVALID_ARG
    assert not h.value
    assert len(built.ggem_last_error(None)) > 0


def test_null_arguments_rejected(built):
    assert built.ggem_plan(None, None, None) == 1
    assert built.ggem_single_layer(None, None, None) == 1
    assert built.ggem_plan_destroy(None) == 0
    # every entry point that takes a plan refuses a NULL one before any device work
    assert built.ggem_set_offgrid(None, 1, 0) == 1
    assert built.ggem_double_layer(None, None, None) == 1
    assert built.ggem_mesh_set(None, 0, None, 0, None) == 1
