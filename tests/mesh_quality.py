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


def tet_metrics(a, b, c, d):
    """Radius ratio gamma = 3 r_in / r_circ and the six dihedral angles
    (degrees) of tetrahedra with vertices a, b, c, d (k x 3), the paper's
    tetrahedral quality measures (Sec. 3.6)."""
    V = np.abs(np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a))) / 6.0
    faces = [(b, c, d), (a, c, d), (a, b, d), (a, b, c)]  # face k is opposite vertex k
    areas = [0.5 * np.linalg.norm(np.cross(q - p, r - p), axis=1) for p, q, r in faces]
    r_in = 3.0 * V / np.sum(areas, axis=0)
    # circumcentre: solve 2 (p_k - a) . x = |p_k|^2 - |a|^2 for k = b, c, d
    M = 2.0 * np.stack([b - a, c - a, d - a], axis=1)
    rhs = np.stack([(b * b).sum(1) - (a * a).sum(1), (c * c).sum(1) - (a * a).sum(1),
                    (d * d).sum(1) - (a * a).sum(1)], axis=1)
    cc = np.linalg.solve(M, rhs[:, :, None])[:, :, 0]
    r_circ = np.linalg.norm(cc - a, axis=1)
    verts = [a, b, c, d]
    # unit normals of the faces, pointing away from the opposite vertex
    normals = []
    for k, (p, q, r) in enumerate(faces):
        n = np.cross(q - p, r - p)
        n /= np.linalg.norm(n, axis=1)[:, None]
        s = np.sign(np.einsum("ij,ij->i", n, p - verts[k]))
        normals.append(n * s[:, None])
    dih = []
    for i in range(4):
        for j in range(i + 1, 4):  # the edge shared by faces i and j
            cosang = -np.einsum("ij,ij->i", normals[i], normals[j])
            dih.append(np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0))))
    return 3.0 * r_in / r_circ, np.stack(dih, axis=1)


def quality3d(pos, col=None, max_edge_factor=2.5, drop_hull=True):
    """Tetrahedral quality of a 3D point set's Delaunay mesh (Sec. 3.6): radius
    ratio average and minimum, dihedral angle extremes, the mean of each
    tetrahedron's smallest dihedral angle, the counts of tetrahedra whose
    smallest dihedral angle is below 10, 20, 30 and 40 degrees, and with
    colours the communication volume (mixed-colour elements / all elements).
    The same filters as quality() drop hull and bridging elements."""
    pos = np.asarray(pos, dtype=np.float64)
    dl = Delaunay(pos)
    tet = dl.simplices
    a, b, c, d = (pos[tet[:, k]] for k in range(4))
    edges = np.stack([np.linalg.norm(p - q, axis=1) for p, q in ((a, b), (a, c), (a, d), (b, c), (b, d), (c, d))],
                     axis=1)
    keep = edges.max(axis=1) < max_edge_factor * np.median(edges) if max_edge_factor else np.ones(len(tet), bool)
    if drop_hull:
        on_hull = np.zeros(len(pos), dtype=bool)
        on_hull[np.unique(dl.convex_hull)] = True
        keep &= ~on_hull[tet].any(axis=1)
    g, dih = tet_metrics(a[keep], b[keep], c[keep], d[keep])
    mins = dih.min(axis=1)
    out = dict(gamma_avg=float(g.mean()), gamma_min=float(g.min()), theta_min=float(dih.min()),
               theta_max=float(dih.max()), theta_min_mean=float(mins.mean()), n_tet=int(keep.sum()),
               slivers={t: int((mins < t).sum()) for t in (10, 20, 30, 40)})
    if col is not None:
        cc = np.asarray(col)[tet[keep]]
        mixed = np.any(cc != cc[:, :1], axis=1)
        out.update(n_et=int(len(cc)), n_eg=int(mixed.sum()))
    return out
