"""Procedural triangle meshes for the TPMC workloads (metres, body frame).

These generators stand in for the paper's Gmsh meshes (§III.C) and spacecraft
models (§III.D), which are not available.  They hold no part of the method's
arithmetic: only vertex positions and triangle indices.  Closed surfaces are
wound counter-clockwise seen from outside (outward normals); open sheets
(plate, solar panels, dish) are two-sided surfaces whose winding only fixes
the sign of their geometric normal.
"""
from __future__ import annotations

import numpy as np


def _finish(xyz, tri):
    return (np.ascontiguousarray(np.asarray(xyz, dtype=np.float64)),
            np.ascontiguousarray(np.asarray(tri, dtype=np.uint32)))


def icosphere(subdivisions: int = 3, radius: float = 1.0):
    """Regular icosahedron subdivided `subdivisions` times; vertices on the sphere.

    20 * 4**subdivisions triangles (1,280 for 3 subdivisions).
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
             (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    F = list(faces)
    for _ in range(subdivisions):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    return _finish(np.array(V) * radius, F)


def plate(size: float = 1.0):
    """Square sheet [-s/2, s/2]^2 in the plane z = 0, two triangles, normal +z."""
    h = size / 2.0
    xyz = [(-h, -h, 0.0), (h, -h, 0.0), (h, h, 0.0), (-h, h, 0.0)]
    return _finish(xyz, [(0, 1, 2), (0, 2, 3)])


def cylinder(radius: float = 0.5, length: float = 2.0, n_azimuth: int = 128, n_axial: int = 15):
    """Closed cylinder along z, centred at the origin.

    Side: n_azimuth x n_axial quads split in two; caps: triangle fans.  The
    default (128, 15) gives 3,840 + 256 = 4,096 triangles.
    """
    ang = 2.0 * np.pi * np.arange(n_azimuth) / n_azimuth
    zs = -length / 2.0 + length * np.arange(n_axial + 1) / n_axial
    xyz = []
    for z in zs:
        for a in ang:
            xyz.append((radius * np.cos(a), radius * np.sin(a), z))
    tri = []
    ring = lambda k, i: k * n_azimuth + (i % n_azimuth)
    for k in range(n_axial):
        for i in range(n_azimuth):
            a, b, c, d = ring(k, i), ring(k, i + 1), ring(k + 1, i + 1), ring(k + 1, i)
            tri += [(a, b, c), (a, c, d)]
    bottom = len(xyz)
    xyz.append((0.0, 0.0, -length / 2.0))
    top = len(xyz)
    xyz.append((0.0, 0.0, length / 2.0))
    for i in range(n_azimuth):
        tri.append((bottom, ring(0, i + 1), ring(0, i)))
        tri.append((top, ring(n_axial, i), ring(n_axial, i + 1)))
    return _finish(xyz, tri)


def _grid_sheet(origin, u, v, nu, nv):
    """Planar grid origin + i/nu u + j/nv v; triangles wound so the normal is u x v."""
    origin, u, v = (np.asarray(a, dtype=np.float64) for a in (origin, u, v))
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
    pts = origin + (ii[..., None] / nu) * u + (jj[..., None] / nv) * v
    xyz = pts.reshape(-1, 3)
    idx = lambda i, j: i * (nv + 1) + j
    tri = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tri += [(a, b, c), (a, c, d)]
    return xyz, np.array(tri, dtype=np.int64)


def _box(lo, hi, cells_per_metre):
    """Closed axis-aligned box, each face a grid; outward winding."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    ext = hi - lo
    parts = []
    for axis in range(3):
        a1, a2 = (axis + 1) % 3, (axis + 2) % 3
        n1 = max(1, int(round(ext[a1] * cells_per_metre)))
        n2 = max(1, int(round(ext[a2] * cells_per_metre)))
        e1 = np.zeros(3); e1[a1] = ext[a1]
        e2 = np.zeros(3); e2[a2] = ext[a2]
        # +axis face: normal e1 x e2 = +axis
        o = lo.copy(); o[axis] = hi[axis]
        parts.append(_grid_sheet(o, e1, e2, n1, n2))
        # -axis face: normal e2 x e1 = -axis
        o = lo.copy()
        parts.append(_grid_sheet(o, e2, e1, n2, n1))
    return parts


def _dish(vertex_x, diameter, focal, n_theta, n_rings):
    """Paraboloid x = vertex_x + rho^2 / (4 f), rho <= diameter / 2, concave side +x."""
    rmax = diameter / 2.0
    xyz = [(vertex_x, 0.0, 0.0)]
    for k in range(1, n_rings + 1):
        rho = rmax * k / n_rings
        for i in range(n_theta):
            a = 2.0 * np.pi * i / n_theta
            xyz.append((vertex_x + rho * rho / (4.0 * focal), rho * np.cos(a), rho * np.sin(a)))
    idx = lambda k, i: 1 + (k - 1) * n_theta + (i % n_theta)
    tri = []
    for i in range(n_theta):
        tri.append((0, idx(1, i), idx(1, i + 1)))
    for k in range(1, n_rings):
        for i in range(n_theta):
            a, b, c, d = idx(k, i), idx(k + 1, i), idx(k + 1, i + 1), idx(k, i + 1)
            tri += [(a, b, c), (a, c, d)]
    return np.array(xyz), np.array(tri, dtype=np.int64)


def _panel(side, cant_deg, span, width, y0, n_span, n_width):
    """Flat 1 x 4 m sheet along +-y from y0, rotated by cant about the y axis."""
    c, s = np.cos(np.radians(cant_deg)), np.sin(np.radians(cant_deg))
    # Before the cant the sheet lies in the y-z plane (normal x); the cant
    # rotates it about its own long axis (the y axis).
    u = np.array([0.0, side * span, 0.0])
    w0 = np.array([0.0, 0.0, width])
    w = np.array([s * w0[2], 0.0, c * w0[2]])  # rotation about y applied to (0, 0, width)
    origin = np.array([0.0, side * y0, 0.0]) - 0.5 * w
    return _grid_sheet(origin, u, w, n_span, n_width)


def satellite(target_triangles: int = 60_000):
    """Concave synthetic satellite.

    * bus: closed box 1 x 1 x 2 m (z long), centred at the origin;
    * two 1 x 4 m two-sided solar panels on +-y, canted +-30 degrees about y;
    * a 1.2 m diameter two-sided paraboloid dish, focal length 0.3 m (0.3 m
      deep), vertex 5 cm in front of the +x face, concave side facing +x.

    About two thirds of the triangles are on the dish.  The default gives
    ~62k triangles; target_triangles=500_000 gives ~500k.
    """
    f = (target_triangles / 62_000.0) ** 0.5
    parts = []
    parts += _box((-0.5, -0.5, -1.0), (0.5, 0.5, 1.0), cells_per_metre=25 * f)
    parts.append(_panel(+1, +30.0, 4.0, 1.0, 0.5, int(round(100 * f)), int(round(25 * f))))
    parts.append(_panel(-1, -30.0, 4.0, 1.0, 0.5, int(round(100 * f)), int(round(25 * f))))
    n_theta = int(round(256 * f))
    n_rings = int(round(78 * f))
    parts.append(_dish(0.55, 1.2, 0.3, n_theta, n_rings))
    xyz, tri, off = [], [], 0
    for X, T in parts:
        xyz.append(np.asarray(X, float))
        tri.append(np.asarray(T) + off)
        off += len(X)
    return _finish(np.concatenate(xyz), np.concatenate(tri))


def hemisphere_shell(radius: float = 1.0, n_lat: int = 32, n_lon: int = 96):
    """Open hemispherical shell z >= 0 (rim on z = 0, pole at +z), two-sided.

    Seen from z < 0 it is a concave cavity facing -z; a flow along +z enters
    it.  n_lon * (2 n_lat - 1) triangles (6,048 for the defaults).
    """
    xyz = [(0.0, 0.0, radius)]
    for i in range(1, n_lat + 1):
        th = 0.5 * np.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * np.pi * j / n_lon
            xyz.append((radius * np.sin(th) * np.cos(ph), radius * np.sin(th) * np.sin(ph), radius * np.cos(th)))
    idx = lambda i, j: 1 + (i - 1) * n_lon + (j % n_lon)
    tri = []
    for j in range(n_lon):
        tri.append((0, idx(1, j), idx(1, j + 1)))
    for i in range(1, n_lat):
        for j in range(n_lon):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tri += [(a, b, c), (a, c, d)]
    return _finish(xyz, tri)


def bounding_sphere(xyz):
    """Centre of the axis-aligned bounding box and the largest vertex distance from it."""
    xyz = np.asarray(xyz, dtype=np.float64)
    c = 0.5 * (xyz.min(axis=0) + xyz.max(axis=0))
    return c, float(np.sqrt(((xyz - c) ** 2).sum(axis=1)).max())


def rotate(xyz, R):
    """Apply a 3x3 matrix to every vertex."""
    return np.ascontiguousarray(np.asarray(xyz, float) @ np.asarray(R, float).T)
