"""Partition borders (host side): the `borders` array of dm_config.

§3.1: the intensity range is cut into n partitions given by integer borders; a uniform
split is the default, and a separate partition for the minimum intensity rho_min of the
volume can help (§3.1, and §4.2 where 32 uniform partitions mix rho_min with visible
intensities of the same partition and lose empty-space skipping).
"""
from __future__ import annotations

import numpy as np


def uniform_borders(N: int, K: int) -> np.ndarray:
    """K+1 lower borders of K equal-width partitions of [0, N): floor(p * N / K)."""
    if not (1 <= K <= N):
        raise ValueError("need 1 <= K <= N")
    return np.array([(p * N) // K for p in range(K + 1)], dtype=np.int32)


def rho_min_borders(N: int, K: int, rho_min: int) -> np.ndarray:
    """Partition 0 = [0, rho_min] (only rho_min occurs in the volume there); the other K-1
    partitions split [rho_min + 1, N) uniformly."""
    if K < 2:
        raise ValueError("a separate rho_min partition needs K >= 2")
    rho_min = int(rho_min)
    rest = N - (rho_min + 1)
    if not (0 <= rho_min < N - 1) or rest < K - 1:
        raise ValueError("rho_min leaves fewer intensities than partitions")
    b = [0] + [rho_min + 1 + (q * rest) // (K - 1) for q in range(K)]
    return np.array(b, dtype=np.int32)
