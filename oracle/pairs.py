"""Image-local qubit pairs (oracle; test infrastructure only).

Sec. II.C assigns the two-qubit observables to horizontal, vertical and
diagonal neighbours of the p x p grid (156 pairs at 7 x 7 instead of the
1,176 all-to-all pairs).  The benchmark pair set is horizontal + vertical.

Order of the list (fixed so that outputs can be compared index by index):
horizontal (r,c)-(r,c+1) row-major by the left pixel, then vertical
(r,c)-(r+1,c) row-major by the top pixel, then (optionally) the diagonal
(r,c)-(r+1,c+1) row-major, then the anti-diagonal (r,c+1)-(r+1,c) row-major.
Each pair is (i, j) with chain indices i < j.
"""
from __future__ import annotations


def image_pairs(p: int, diagonals: bool = False) -> list:
    idx = lambda r, c: r * p + c  # noqa: E731  row-major flattening (Sec. II.B)
    pairs = []
    for r in range(p):
        for c in range(p - 1):
            pairs.append((idx(r, c), idx(r, c + 1)))
    for r in range(p - 1):
        for c in range(p):
            pairs.append((idx(r, c), idx(r + 1, c)))
    if diagonals:
        for r in range(p - 1):
            for c in range(p - 1):
                pairs.append((idx(r, c), idx(r + 1, c + 1)))
        for r in range(p - 1):
            for c in range(p - 1):
                pairs.append((idx(r, c + 1), idx(r + 1, c)))
    return pairs
