"""Shared helpers for the tests (not product code)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def mask_to_mu(mask_words: np.ndarray, nnb: int) -> np.ndarray:
    """[W][N] int32 bit mask -> [N][nnb] uint8 (1 = intact)."""
    m = mask_words.astype(np.int64) & 0xFFFFFFFF
    N = m.shape[1]
    mu = np.zeros((N, nnb), dtype=np.uint8)
    for k in range(nnb):
        mu[:, k] = (m[k >> 5] >> (k & 31)) & 1
    return mu


def mu_to_mask(mu: np.ndarray) -> np.ndarray:
    """[N][nnb] uint8 -> [W][N] int32 bit mask."""
    N, nnb = mu.shape
    W = (nnb + 31) // 32
    m = np.zeros((W, N), dtype=np.int64)
    for k in range(nnb):
        m[k >> 5] |= (mu[:, k].astype(np.int64) & 1) << (k & 31)
    m = np.where(m >= 2 ** 31, m - 2 ** 32, m)
    return m.astype(np.int32)
