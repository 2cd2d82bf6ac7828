"""Query pairs: (v, w) drawn uniformly from V x V with replacement (the paper's Sec. 5
uses random sources and random targets)."""

from __future__ import annotations

import numpy as np


def random_pairs(n: int, q: int, seed: int) -> np.ndarray:
    """int32[q, 2] uniform random vertex pairs (with replacement; v == w allowed)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, size=(q, 2), dtype=np.int64).astype(np.int32)
