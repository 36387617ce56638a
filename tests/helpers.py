"""Shared helpers of the GPU parity tests."""
import numpy as np


def rel_l1(got, want) -> float:
    """||got - want||_1 / ||want||_1 (the parity metric for float storage)."""
    g = np.asarray(got, dtype=np.float64).ravel()
    w = np.asarray(want, dtype=np.float64).ravel()
    return float(np.abs(g - w).sum() / np.abs(w).sum())


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_host(t) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)
