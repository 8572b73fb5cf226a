"""Front-to-back order of the K subsets' cells for one view (Sec. 4.2, saturation skipping).

The subsets are the cells of a k-d partition (axis-aligned boxes, infinite on unsplit
sides).  A binary space partition gives a visibility order: at each split plane the cells
on the camera's side come first.  The order is recovered from the cells alone: a set of
cells is split by an axis-aligned plane that puts every cell entirely on one side (the
first such plane over the axes x, y, z and ascending coordinates), the side holding the
camera centre is ordered first, and both sides are ordered the same way.
"""
from __future__ import annotations

import math

import numpy as np


def front_to_back(boxes, eye) -> list[int]:
    """Indices of the cells `boxes` ([K, 2, 3]: lo, hi) in front-to-back order from `eye`."""
    b = np.asarray(boxes, np.float64)
    e = np.asarray(eye, np.float64)

    def split(ids):
        for ax in range(3):
            planes = sorted({float(b[i, s, ax]) for i in ids for s in (0, 1)
                             if math.isfinite(float(b[i, s, ax]))})
            for p in planes:
                below = [i for i in ids if b[i, 1, ax] <= p]
                above = [i for i in ids if b[i, 0, ax] >= p]
                if below and above and len(below) + len(above) == len(ids):
                    return (below, above) if e[ax] <= p else (above, below)
        return None

    def order(ids):
        if len(ids) <= 1:
            return list(ids)
        parts = split(ids)
        if parts is None:
            raise ValueError("the boxes are not the cells of a k-d partition")
        return order(parts[0]) + order(parts[1])

    return order(list(range(b.shape[0])))


def orders_for_views(boxes, cams) -> np.ndarray:
    """[V, K] int32 front-to-back subset order of every camera."""
    return np.array([front_to_back(boxes, c.eye) for c in cams], np.int32)
