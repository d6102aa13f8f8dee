"""Droplet statistics of a density field, for the oracle side of the condensation
comparisons.  TEST INFRASTRUCTURE ONLY (tests and bench legs that use the oracle).

The measure (the reading of the droplet measure for the channel of Section 3.3):
liquid nodes have rho above a threshold; droplets are 8-connected liquid components
that touch a wall row (y = 0 bottom, y = ny - 1 top; a component touching both
counts for both); a droplet's position is the mean x of its nodes (the circular mean
when x is periodic); the spacing on a wall is the mean distance between neighbouring
positions, (last - first) / (count - 1), or nx / count with periodic x; the
condensed mass is the sum of rho - rho_v over liquid nodes.  Component labelling is
scipy's ndimage.label with the full 3 x 3 structure; periodic x joins the labels
that meet across the seam.
"""
from __future__ import annotations

import numpy as np


def contact_angle(rho: np.ndarray, rho_mid: float) -> float:
    """Contact angle of a sessile cap on the bottom wall (wall at y = -1/2): 2 atan(2h / w)
    from the cap height h on its centre column and the base width w along row 0, both with
    linear interpolation of the rho_mid crossing (the reading of the droplet measure)."""
    row = rho[0]
    xs = np.where(row > rho_mid)[0]
    if xs.size == 0:
        return 180.0  # the drop has lifted off the wall
    if xs.size == row.size:
        return 0.0  # a film covers the wall
    x0, x1 = xs.min(), xs.max()
    left = x0 - (row[x0] - rho_mid) / (row[x0] - row[x0 - 1])
    right = x1 + (row[x1] - rho_mid) / (row[x1] - row[x1 + 1])
    w = right - left
    c = int(round(0.5 * (x0 + x1)))
    colv = rho[:, c]
    ys = np.where(colv > rho_mid)[0]
    y1 = ys.max()
    h = y1 + (colv[y1] - rho_mid) / (colv[y1] - colv[y1 + 1]) + 0.5
    return float(np.degrees(2 * np.arctan(2 * h / w)))


def droplet_stats(rho: np.ndarray, threshold: float, rho_v: float,
                  periodic_x: bool = False) -> dict:
    from scipy import ndimage
    rho = np.asarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    liq = rho > threshold
    lab, n = ndimage.label(liq, structure=np.ones((3, 3), dtype=int))
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    if periodic_x and nx > 1:
        for y in range(ny):
            for dy in (-1, 0, 1):
                y2 = y + dy
                if 0 <= y2 < ny and lab[y, nx - 1] and lab[y2, 0]:
                    a, b = find(lab[y, nx - 1]), find(lab[y2, 0])
                    if a != b:
                        parent[max(a, b)] = min(a, b)
    roots = np.array([find(k) for k in range(n + 1)])
    comp = roots[lab]
    positions = {0: [], 1: []}
    detached = 0
    for c in np.unique(comp[liq]):
        ys, xs = np.nonzero(comp == c)
        if periodic_x:
            ang = np.arctan2(np.sin(2 * np.pi * xs / nx).sum(), np.cos(2 * np.pi * xs / nx).sum())
            pos = (ang % (2 * np.pi)) * nx / (2 * np.pi)
        else:
            pos = xs.mean()
        bottom, top = (ys == 0).any(), (ys == ny - 1).any()
        if bottom:
            positions[0].append(pos)
        if top:
            positions[1].append(pos)
        if not bottom and not top:
            detached += 1
    spacing = []
    for w in (0, 1):
        p = sorted(positions[w])
        if len(p) < 2:
            spacing.append(0.0)
        elif periodic_x:
            spacing.append(nx / len(p))
        else:
            spacing.append((p[-1] - p[0]) / (len(p) - 1))
    return {"count": [len(positions[0]), len(positions[1])], "spacing": spacing,
            "condensed_mass": float((rho[liq] - rho_v).sum()), "liquid_nodes": int(liq.sum()),
            "detached": detached}
