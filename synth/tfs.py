"""Seeded synthetic 1D RGBA transfer functions and TF-edit sequences.

The paper times the update on six hand-made TFs (TF1-TF6, §4.2, Table 1) that do not ship
with it.  These generators stand in for them: 1-3 piecewise-linear opacity ramps (tents or
trapezoids) over the N-entry intensity domain, then edits that move a ramp and rescale its
width, as a user dragging TF widgets would.  Opacity is computed in float32 and is exactly
0.0 outside the ramps.  Special TFs (all-zero, all-visible, one intensity, and TFs whose
visible set is a union of whole partitions) cover the method's degenerate cases.

This module only draws inputs; it holds none of the method's arithmetic.  A TF is an
(N, 4) float32 numpy array, entry i mapping intensity i to (R, G, B, A).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Ramp:
    centre: float
    width: float
    peak: float
    trapezoid: bool


def _colour(N: int) -> np.ndarray:
    t = np.linspace(0.0, 1.0, N, dtype=np.float32)
    return np.stack([t, 0.5 + 0.5 * np.sin(6.0 * t).astype(np.float32), 1.0 - t], 1)


def tf_from_ramps(N: int, ramps) -> np.ndarray:
    i = np.arange(N, dtype=np.float32)
    alpha = np.zeros(N, dtype=np.float32)
    for r in ramps:
        half = np.float32(r.width * 0.5)
        d = np.abs(i - np.float32(r.centre))
        if r.trapezoid:
            # flat top over the inner half of the support
            a = np.clip((half - d) / np.float32(max(half * 0.5, 1e-3)), 0.0, 1.0)
        else:
            a = np.clip(1.0 - d / np.float32(max(half, 1e-3)), 0.0, 1.0)
        a = (a * np.float32(r.peak)).astype(np.float32)
        a[d >= half] = 0.0
        alpha = np.maximum(alpha, a)
    tf = np.empty((N, 4), dtype=np.float32)
    tf[:, :3] = _colour(N)
    tf[:, 3] = alpha
    return tf


def random_ramps(rng: np.random.Generator, N: int):
    n = int(rng.integers(1, 4))
    return [Ramp(centre=float(rng.uniform(0, N)),
                 width=float(rng.uniform(N / 32, N / 4)),
                 peak=float(rng.uniform(0.1, 1.0)),
                 trapezoid=bool(rng.integers(0, 2)))
            for _ in range(n)]


def tf_edit_sequence(seed: int, N: int, count: int):
    """`count` TFs: a random start, then each edit moves one ramp's centre by
    U[-N/16, N/16] and scales its width by U[0.7, 1.4] (width kept in [2, N/2])."""
    rng = np.random.default_rng(seed)
    ramps = random_ramps(rng, N)
    out = []
    for _ in range(count):
        k = int(rng.integers(0, len(ramps)))
        r = ramps[k]
        c = float(np.clip(r.centre + rng.uniform(-N / 16, N / 16), 0, N - 1))
        w = float(np.clip(r.width * rng.uniform(0.7, 1.4), 2.0, N / 2))
        ramps[k] = Ramp(c, w, r.peak, r.trapezoid)
        out.append(tf_from_ramps(N, ramps))
    return out


def zero_tf(N: int) -> np.ndarray:
    tf = np.zeros((N, 4), dtype=np.float32)
    tf[:, :3] = _colour(N)
    return tf


def all_visible_tf(N: int, alpha: float = 0.5) -> np.ndarray:
    tf = zero_tf(N)
    tf[:, 3] = np.float32(alpha)
    return tf


def single_intensity_tf(N: int, i: int, alpha: float = 1.0) -> np.ndarray:
    tf = zero_tf(N)
    tf[i, 3] = np.float32(alpha)
    return tf


def uniform_borders(N: int, K: int) -> np.ndarray:
    """Lower borders of K equal-width partitions of [0, N) plus the end, floor(p*N/K)."""
    return np.array([(p * N) // K for p in range(K + 1)], dtype=np.int32)


def aligned_tf(seed: int, N: int, borders: np.ndarray, frac: float = 0.4) -> np.ndarray:
    """A TF whose visible intensities are a random union of whole partitions: every
    partition is either all visible or all invisible (alpha varies inside it)."""
    rng = np.random.default_rng(seed)
    K = len(borders) - 1
    tf = zero_tf(N)
    for p in range(K):
        if rng.uniform() < frac:
            lo, hi = int(borders[p]), int(borders[p + 1])
            tf[lo:hi, 3] = rng.uniform(0.05, 1.0, size=hi - lo).astype(np.float32)
    return tf


def special_tfs(N: int, borders: np.ndarray, seed: int = 7):
    """The degenerate TFs every config is also checked on."""
    out = [zero_tf(N), all_visible_tf(N), single_intensity_tf(N, N // 3),
           single_intensity_tf(N, 0), single_intensity_tf(N, N - 1)]
    out += [aligned_tf(seed + k, N, borders) for k in range(10)]
    nan_tf = zero_tf(N)
    nan_tf[N // 2, 3] = np.float32("nan")      # NaN opacity is not "non-zero alpha"
    nan_tf[N // 4, 3] = np.float32(-0.0)
    out.append(nan_tf)
    return out
