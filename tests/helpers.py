"""Shared test helpers: the parity metric and GPU plumbing."""
import numpy as np

# Bar for FP32 GPU results against the FP64 oracle (max relative error, rel_err below).
TOL = 1e-4


def rel_err(got, ref):
    """max over pixels and channels of |got - ref| / max(|ref|, 0.01 * RMS(ref)).

    The floor keeps near-zero reference values (dark pixels) from dominating: an error is
    measured relative to the local value, but never relative to less than 1% of the
    image's RMS.
    """
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = 0.01 * np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0
    denom = np.maximum(np.abs(ref), max(floor, 1e-30))
    return float(np.max(np.abs(got - ref) / denom)) if ref.size else 0.0


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
