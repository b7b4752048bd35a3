"""Sub-blocks that contain a node's whole dependency cone for one step.

One Cash-Karp step changes x at a node through the six stage derivatives
there; stage s at a node reads the stage input y_s within index distance 2
(B at the six neighbours, and B at a node needs x at its own neighbours),
and y_s at a node combines x and k_1..k_{s-1} at that node only.  So the
updated x at node n depends on the step's starting x (and B0) within index
distance 12 (6 stages x 2) and on nothing else.  An oracle step on a
sub-block whose artificial faces (those not on the grid's own boundary) lie
at least RADIUS nodes from n therefore gives n's updated x exactly as a
step on the whole grid would -- which lets a grid too large for the CPU
oracle be checked node by node.  The property itself is checked on the CPU
against whole-grid oracle steps (tests/test_cone_subblock.py).

Wrong values enter at the artificial faces (held fixed, one-sided
differences there) and move inward by 2 nodes per stage: after six stages
they stop 2 nodes short of distance 12 -- RADIUS 14 leaves margin.
"""
from __future__ import annotations

from dataclasses import dataclass

RADIUS = 14


@dataclass(frozen=True)
class SubGrid:
    """Node counts and the parent grid's label spacings (taken over exactly,
    not recomputed from the sub-block's extent, so that the oracle sees the
    same h to the last bit)."""
    nx: int
    ny: int
    nz: int
    h: tuple


def subblock(g, x, B0, i, j, k, radius=RADIUS):
    """(sub-grid, x, B0, (i, j, k) within the sub-block) around node (i, j, k);
    faces on the grid's own boundary stay where they are."""
    lo_i = [max(0, c - radius) for c in (i, j, k)]
    hi_i = [min(n - 1, c + radius) for c, n in zip((i, j, k), (g.nx, g.ny, g.nz))]
    sub = SubGrid(hi_i[0] - lo_i[0] + 1, hi_i[1] - lo_i[1] + 1, hi_i[2] - lo_i[2] + 1,
                  tuple(g.h))
    sl = (slice(None), slice(lo_i[2], hi_i[2] + 1), slice(lo_i[1], hi_i[1] + 1),
          slice(lo_i[0], hi_i[0] + 1))
    return sub, x[sl].copy(), B0[sl].copy(), (i - lo_i[0], j - lo_i[1], k - lo_i[2])
