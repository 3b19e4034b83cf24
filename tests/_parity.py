"""Comparison helper of the GPU parity tests."""
import numpy as np


def assert_close(a, b, tol):
    """GPU result a against the oracle's b: the max-norm relative error
    max|a - b| / max|b| below tol, and, so that small components are held to
    account as well, the relative error of every component larger than 1e-3
    of the largest below 500 tol (the max-norm bound alone would allow
    1000 tol there)."""
    a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    b = np.asarray(b)
    m = np.abs(b).max()
    e = np.abs(a - b)
    assert e.max() < tol * m, f"max-norm relative error {e.max() / m:.3e} >= {tol:.1e}"
    big = np.abs(b) > 1e-3 * m
    el = float((e[big] / np.abs(b[big])).max()) if big.any() else 0.0
    assert el < 500 * tol, f"per-component relative error {el:.3e} >= {500 * tol:.1e}"
    return e.max() / m, el
