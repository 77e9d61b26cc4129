"""Block averaging for the statistical pins."""
import numpy as np


def block_mean(x, n_blocks=20):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // n_blocks * n_blocks
    b = x[:n].reshape(n_blocks, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(n_blocks))
