"""Per-point cost model of Sec. 2.3 (Table 1, lower bound row) and
Sec. 3.1.2 (the SPIDER_C / SPIDER_I / SPIDER_P formulas, Table 2) --
TEST INFRASTRUCTURE ONLY.

The formulas are for a Box-2D stencil of radius r on an A x B grid, with
c x c points updated per tile.  Dividing by A*B gives per-point figures.

Table 2 prints 56 computation operations for SPIDER at r = 3, c = 8.  The
formula with the ceiling on (2r+c)/4 gives 64; without that ceiling it gives
56 = (2r+1)(2r+2), the MAC count of L = 2r+2 outputs times 2r+1 kernel rows
with half of the 2L-wide padded row skipped.  ``spider_costs`` therefore
exposes the ceiling as a switch; the input and parameter counts of Table 2
(14 and 7) match the formula with the ceiling.
"""
from __future__ import annotations

import math


def lower_bound(r: int, c: int):
    """Table 1, "Lower Bound" row, per point: (MACs, input, parameter accesses)."""
    return ((2 * r + 1) ** 2, (c + 2 * r) ** 2 / c ** 2, (2 * r + 1) ** 2 / c ** 2)


def spider_costs(r: int, c: int, ceil_compute: bool = True):
    """Sec. 3.1.2 formulas, per point: (computation, input, parameter)."""
    g = math.ceil((2 * r + c) / 4)
    gc = g if ceil_compute else (2 * r + c) / 4
    cc = math.ceil(c / 8)
    comp = 256 / c ** 2 * (r + 1) * cc ** 2 * gc
    inp = 32 / c ** 2 * (2 * r + 1) * cc * g
    par = 16 / c ** 2 * (2 * r + 1) * cc * g
    return comp, inp, par
