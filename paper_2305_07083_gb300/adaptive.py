"""Variance-driven work distribution for image-parallel rendering.

Sec. 4.1.1: tiles can be rendered redundantly by several ranks with
different seeds and averaged by the tile operation (DFB_AVERAGE); tiles with
a higher variance get more renders.  The per-tile variance comes from the
framebuffer (dfb_read_variance); this module only turns it into render
counts on the host.
"""

from __future__ import annotations

import numpy as np


def redundancy(tile_variance, k_min: int = 1, k_max: int = 8) -> np.ndarray:
    """Renders per tile for the next pass: k_min for a tile at or below the
    median variance, growing with the ratio to the median, capped at k_max.
    Deterministic and monotone in the variance."""
    v = np.nan_to_num(np.asarray(tile_variance, dtype=np.float64), nan=0.0)
    if k_min < 1 or k_max < k_min:
        raise ValueError("need 1 <= k_min <= k_max")
    med = float(np.median(v)) if v.size else 0.0
    if med <= 0.0:
        ratio = np.where(v > 0.0, float(k_max), 1.0)
    else:
        ratio = np.maximum(v / med, 1.0)
    return np.clip(np.ceil(k_min * ratio), k_min, k_max).astype(np.int64)
