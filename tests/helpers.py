"""Shared helpers of the test suite (no method arithmetic)."""
import numpy as np


def rel_l2(a, b):
    """Per-field relative L2 distance of two (3, ncoef) spectral states (numpy complex)."""
    a = np.asarray(a)
    b = np.asarray(b)
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=-1))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=-1))
    return num / np.where(den > 0, den, 1.0)


def to_numpy(t):
    return t.detach().cpu().numpy()
