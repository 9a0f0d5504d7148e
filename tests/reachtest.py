"""Shared helpers of the test suite: tolerances and GPU availability."""
import numpy as np

# FP64 bounds: |g - o| <= 1e-10 max(|o|, s), s = max_i |o_i| (a per-vector floor
# so that bounds near zero are compared on the scale of the vector)
TOL64 = 1e-10
# FP32 Monte Carlo trajectories against the FP64 oracle on the same samples
TOL32 = 1e-4


def assert_close(g, o, tol, what=""):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    s = np.abs(o).max() if o.size else 0.0
    err = np.abs(g - o)
    lim = tol * np.maximum(np.abs(o), s)
    bad = np.flatnonzero(err > lim)
    assert bad.size == 0, (f"{what}: {bad.size} of {o.size} outside tolerance {tol}; first at "
                           f"{bad[0]}: gpu {g.flat[bad[0]]!r} oracle {o.flat[bad[0]]!r}")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
