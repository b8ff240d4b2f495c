"""Voronoi cells by brute-force half-plane clipping (independent reference for
the tessellation and geometry pins; numpy only)."""
import numpy as np


def clip(poly, a, b):
    """Keep the part of polygon poly (k,2) with a.x <= b."""
    out = []
    k = len(poly)
    for i in range(k):
        p, q = poly[i], poly[(i + 1) % k]
        fp, fq = a @ p - b, a @ q - b
        if fp <= 0:
            out.append(p)
        if (fp < 0 < fq) or (fq < 0 < fp):
            t = fp / (fp - fq)
            out.append(p + t * (q - p))
    return np.array(out)


def polygon_area_centroid(poly):
    x, y = poly[:, 0], poly[:, 1]
    xs, ys = np.roll(x, -1), np.roll(y, -1)
    cr = x * ys - xs * y
    A = 0.5 * cr.sum()
    cx = ((x + xs) * cr).sum() / (6 * A)
    cy = ((y + ys) * cr).sum() / (6 * A)
    return A, cx, cy


def voronoi_cells(x, y, box, periodic):
    x0, x1, y0, y1 = box
    Lx, Ly = x1 - x0, y1 - y0
    pts = np.stack([x, y], 1)
    if periodic:
        imgs = [pts + np.array([sx * Lx, sy * Ly]) for sx in (-1, 0, 1) for sy in (-1, 0, 1)]
        others = np.concatenate(imgs)
    else:
        others = pts
    res = []
    for i, p in enumerate(pts):
        if periodic:
            poly = p + np.array([[-Lx, -Ly], [Lx, -Ly], [Lx, Ly], [-Lx, Ly]], float)
        else:
            poly = np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], float)
        for q in others:
            if np.all(q == p):
                continue
            a = q - p
            b = 0.5 * (q @ q - p @ p)
            poly = clip(poly, a, b)
        res.append(polygon_area_centroid(poly))
    return np.array(res)
