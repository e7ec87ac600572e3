"""FP64 CPU oracle of the connectivity loss (Sec. 4 / appendix, L_connect).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For cell i with bound radius R_i and site p_i, over the listed neighbours j
(the neighbour lists stand in for the Cech adjacency; pairs whose spheres do
not overlap add nothing):

    L_connect(i) = sum_j max(R_i + R_j - |p_i - p_j|, 0)^2

and the gradient of L = sum_i L_connect(i), with o = R_i + R_j - d > 0 and
d = |p_i - p_j|:  dL/dR_i += 2 o, dL/dR_j += 2 o, dL/dp_i += 2 o (p_j - p_i)/d,
dL/dp_j -= 2 o (p_j - p_i)/d.  Plain loops in double precision.
"""
from __future__ import annotations

import math

import numpy as np


def connect(pos, R, nbr):
    """Per-cell loss [N] and the gradients (dL/dpos [N,3], dL/dR [N]) of
    their sum."""
    pos = np.asarray(pos, np.float64)
    R = np.asarray(R, np.float64)
    nbr = np.asarray(nbr)
    n = pos.shape[0]
    loss = np.zeros(n)
    gpos = np.zeros((n, 3))
    gR = np.zeros(n)
    for i in range(n):
        for j in nbr[i]:
            j = int(j)
            if j < 0 or j >= n or j == i:
                continue
            a = pos[j] - pos[i]
            d = math.sqrt(float(a @ a))
            o = R[i] + R[j] - d
            if o <= 0.0:
                continue
            loss[i] += o * o
            gR[i] += 2 * o
            gR[j] += 2 * o
            if d > 0.0:
                gpos[i] += 2 * o * a / d
                gpos[j] -= 2 * o * a / d
    return loss, gpos, gR


def cech_lists(pos, R):
    """The Cech adjacency of the bounding spheres (Sec. 3.3): for each cell,
    every other cell whose sphere overlaps its own, |p_i - p_j| < R_i + R_j,
    by brute force over all pairs (lists padded with -1)."""
    pos = np.asarray(pos, np.float64)
    R = np.asarray(R, np.float64)
    n = pos.shape[0]
    rows = []
    for i in range(n):
        d = np.sqrt(((pos - pos[i]) ** 2).sum(1))
        js = np.nonzero((d < R[i] + R) & (np.arange(n) != i))[0]
        rows.append(js)
    k = max((len(r) for r in rows), default=0)
    out = np.full((n, k), -1, np.int64)
    for i, r in enumerate(rows):
        out[i, :len(r)] = r
    return out


def connect_cech(pos, R):
    """L_connect over the exact Cech adjacency (the paper's definition):
    `connect` applied to `cech_lists`."""
    return connect(pos, R, cech_lists(pos, R))
