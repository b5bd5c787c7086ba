"""Zone partition oracle for large-scale scenes.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: used only by tests and the
benchmark's CPU-baseline leg; it never imports the CUDA package.

Sec. III-A ("Support Large-scale Scenes"): sensor frames are clustered by
their XY location into 40 x 40 m zones, with 25 % relative padding, and
while rendering two threads double-buffer the zones, swapping in the
Gaussians of the next block as the vehicle moves.  Reading of the points the
paper leaves open:
  grid     zone (i, j) is the square [x0 + i s, x0 + (i+1) s) x
           [y0 + j s, y0 + (j+1) s), s = zone size, id = j nx + i;
  padding  a surfel belongs to a zone when its centre lies in the square
           grown by padding x s on every side (so up to four zones);
  vehicle  the zone of a point is the unpadded square holding it.
"""
from __future__ import annotations

import math

import numpy as np


def zone_of(grid, x, y):
    """Zone id of a point (unpadded square), -1 outside the grid."""
    i = math.floor((x - grid["x0"]) / grid["zone_size"])
    j = math.floor((y - grid["y0"]) / grid["zone_size"])
    if 0 <= i < grid["nx"] and 0 <= j < grid["ny"]:
        return j * grid["nx"] + i
    return -1


def members(grid, pos):
    """Per zone id, the ascending indices of the surfels whose centre lies in
    the zone's padded square (brute force over every zone and surfel)."""
    s, p = grid["zone_size"], grid["padding"]
    x, y = np.asarray(pos, np.float64)[:, 0], np.asarray(pos, np.float64)[:, 1]
    out = []
    for j in range(grid["ny"]):
        for i in range(grid["nx"]):
            lo_x, hi_x = grid["x0"] + (i - p) * s, grid["x0"] + (i + 1 + p) * s
            lo_y, hi_y = grid["y0"] + (j - p) * s, grid["y0"] + (j + 1 + p) * s
            inside = (x >= lo_x) & (x < hi_x) & (y >= lo_y) & (y < hi_y)
            out.append(np.nonzero(inside)[0])
    return out
