"""Element-wise parity check shared by the GPU tests."""
import numpy as np

# FP64 bar: |x - y| <= 1e-13 + 1e-11 |y| per element (y = oracle)
ATOL = 1e-13
RTOL = 1e-11


def check(got, ref, atol=ATOL, rtol=RTOL, what=""):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    excess = np.abs(got - ref) - (atol + rtol * np.abs(ref))
    if np.any(excess > 0):
        i = np.unravel_index(np.argmax(excess), excess.shape)
        raise AssertionError(f"{what}: {int(np.sum(excess > 0))} elements out of tolerance; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} diff {got[i] - ref[i]:.3e}")


def report(got, ref):
    d = np.abs(np.asarray(got) - np.asarray(ref))
    r = d / np.maximum(np.abs(ref), 1e-300)
    big = np.abs(ref) > 1e-3 * np.max(np.abs(ref))
    return {"max_abs": float(d.max()), "max_rel_significant": float(r[big].max()) if big.any() else 0.0,
            "median_abs": float(np.median(d))}
