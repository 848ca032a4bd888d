"""Per-bubble migration velocity and position of Sec. 4.3, the plain way.

TEST INFRASTRUCTURE: the definition the library's device labelling is checked
against.  Only tests, the smoke check and the benchmark's CPU-baseline leg may use it;
it does not import the CUDA package.

Sec. 4.3 defines, for the bubble alpha (a connected region where phi < 0),
    u_b = sum_{phi_alpha < 0} u_x phi / sum_{phi_alpha < 0} phi,
    x_b = sum_{phi_alpha < 0} x phi   / sum_{phi_alpha < 0} phi
(integrals over the region written as node sums, dx = 1).  The paper does not say how
regions are told apart; here they are the 4-connected components of phi < 0, wrapping
along periodic axes, found by breadth-first flood fill.  Coordinates along a periodic
axis are taken at each node's image nearest to the region's first node (lowest row,
then lowest column), and the centroid is reported modulo the lattice size.
"""
from __future__ import annotations

from collections import deque

import numpy as np

KEYS = ("nodes", "sum_phi", "u_b", "v_b", "x_b", "y_b")


def label(phi, periodic_x=False, periodic_y=False):
    """Component index of every node (-1 where phi >= 0), components numbered in the
    order of their first node (row-major), and the list of first nodes (y, x)."""
    ny, nx = phi.shape
    lab = np.full((ny, nx), -1, dtype=np.int64)
    firsts = []
    inside = phi < 0
    for y0, x0 in zip(*np.nonzero(inside)):
        if lab[y0, x0] >= 0:
            continue
        k = len(firsts)
        firsts.append((int(y0), int(x0)))
        lab[y0, x0] = k
        queue = deque([(int(y0), int(x0))])
        while queue:
            y, x = queue.popleft()
            for qy, qx in ((y, x + 1), (y, x - 1), (y + 1, x), (y - 1, x)):
                if periodic_x:
                    qx %= nx
                if periodic_y:
                    qy %= ny
                if 0 <= qx < nx and 0 <= qy < ny and inside[qy, qx] and lab[qy, qx] < 0:
                    lab[qy, qx] = k
                    queue.append((qy, qx))
    return lab, firsts


def bubbles(phi, ux, uy, periodic_x=False, periodic_y=False):
    """List of dicts (KEYS) per bubble, ordered by x_b then y_b, sums in FP64."""
    phi = np.asarray(phi, dtype=np.float64)
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    ny, nx = phi.shape
    lab, firsts = label(phi, periodic_x, periodic_y)
    out = []
    for k, (y0, x0) in enumerate(firsts):
        ys, xs = np.nonzero(lab == k)
        dx = xs - x0
        dy = ys - y0
        if periodic_x:
            dx = np.where(dx > nx // 2, dx - nx, np.where(dx < -(nx // 2), dx + nx, dx))
        if periodic_y:
            dy = np.where(dy > ny // 2, dy - ny, np.where(dy < -(ny // 2), dy + ny, dy))
        p = phi[ys, xs]
        s = p.sum()
        xb = x0 + (p * dx).sum() / s
        yb = y0 + (p * dy).sum() / s
        if periodic_x:
            xb %= nx
        if periodic_y:
            yb %= ny
        out.append(dict(nodes=float(len(xs)), sum_phi=float(s), u_b=float((p * ux[ys, xs]).sum() / s),
                        v_b=float((p * uy[ys, xs]).sum() / s), x_b=float(xb), y_b=float(yb)))
    out.sort(key=lambda b: (b["x_b"], b["y_b"]))
    return out
