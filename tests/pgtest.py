"""Helpers shared by the GPU parity tests."""

import numpy as np
import pytest

# Newton tolerances (per-particle relative error against the FP64 oracle)
MEDIAN_TOL = 2e-6
MAX_TOL = 1e-4


def rel_vec(a, ref):
    return np.linalg.norm(np.asarray(a) - np.asarray(ref), axis=1) / np.linalg.norm(ref, axis=1)


def rel_scalar(p, ref):
    return np.abs(np.asarray(p) - np.asarray(ref)) / np.abs(ref)


def assert_parity(err, median_tol=MEDIAN_TOL, max_tol=MAX_TOL, what="a"):
    med, mx = float(np.median(err)), float(np.max(err))
    assert med <= median_tol and mx <= max_tol, f"{what}: median {med:.3e} max {mx:.3e}"
    return med, mx


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1203_4037_gb300 as pg
    pg.build()
    return pg
