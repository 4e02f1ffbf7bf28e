"""Post-hoc triangulation quality of a 2D point set (the paper's mesh-quality
criterion for triangles, Sec. 4: G = 2 sqrt(3) S / (P H) with S the area, P the
half-perimeter and H the longest edge; the triangle angles). The points are
triangulated with scipy's Delaunay; triangles with a vertex on the convex hull
(boundary slivers) or an edge much longer than the typical one (bridges over a
hole or a concave part of the region) are left out, the same way for every
point set compared."""
import numpy as np
from scipy.spatial import Delaunay


def triangle_metrics(a, b, c):
    """G and the three angles (degrees) of triangles with vertices a, b, c (k x 2)."""
    la = np.linalg.norm(b - c, axis=1)
    lb = np.linalg.norm(c - a, axis=1)
    lc = np.linalg.norm(a - b, axis=1)
    S = 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    P = 0.5 * (la + lb + lc)
    H = np.maximum(np.maximum(la, lb), lc)
    G = 2.0 * np.sqrt(3.0) * S / (P * H)
    def ang(x, y, z):  # angle opposite side x
        return np.degrees(np.arccos(np.clip((y * y + z * z - x * x) / (2 * y * z), -1.0, 1.0)))
    A = np.stack([ang(la, lb, lc), ang(lb, lc, la), ang(lc, la, lb)], axis=1)
    return G, A


def quality(pos, col=None, max_edge_factor=2.5, drop_hull=True):
    """G_avg, G_min, theta_min, theta_max, mean of each triangle's smallest
    angle, count of triangles with an angle < 30 degrees, share of angles in
    [55, 65] degrees, triangle count; with colours, also the communication
    volume of the partition (Sec. 4): N_eg / N_et, N_eg the kept elements
    (triangles) with vertices of different colours and N_et all kept elements.
    max_edge_factor None keeps triangles of any size (convex regions whose
    resolution varies strongly, where a long edge is no sign of a bridge)."""
    pos = np.asarray(pos, dtype=np.float64)
    dl = Delaunay(pos)
    tri = dl.simplices
    on_hull = np.zeros(len(pos), dtype=bool)
    on_hull[np.unique(dl.convex_hull)] = True
    a, b, c = pos[tri[:, 0]], pos[tri[:, 1]], pos[tri[:, 2]]
    edges = np.concatenate([np.linalg.norm(a - b, axis=1), np.linalg.norm(b - c, axis=1),
                            np.linalg.norm(c - a, axis=1)])
    med = np.median(edges)
    longest = np.maximum(np.maximum(np.linalg.norm(a - b, axis=1), np.linalg.norm(b - c, axis=1)),
                         np.linalg.norm(c - a, axis=1))
    keep = longest < max_edge_factor * med if max_edge_factor else np.ones(len(tri), dtype=bool)
    if drop_hull:
        keep &= ~on_hull[tri].any(axis=1)
    G, A = triangle_metrics(a[keep], b[keep], c[keep])
    extra = {}
    if col is not None:
        c = np.asarray(col)[tri[keep]]
        mixed = (c[:, 0] != c[:, 1]) | (c[:, 1] != c[:, 2])
        extra = dict(n_et=int(len(c)), n_eg=int(mixed.sum()))
    return dict(**extra, G_avg=float(G.mean()), G_min=float(G.min()), theta_min=float(A.min()), theta_max=float(A.max()),
                theta_min_mean=float(A.min(axis=1).mean()), n_lt30=int((A.min(axis=1) < 30.0).sum()),
                share_55_65=float(((A >= 55.0) & (A <= 65.0)).mean()), n_tri=int(keep.sum()))
