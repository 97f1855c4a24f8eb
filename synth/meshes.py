"""Deterministic closed triangle meshes (vertices in metres, wavelength 1).

Every generator returns ``(xyz, tri)``: ``xyz`` float64 (n_vert, 3) and
``tri`` int32 (n_tri, 3) with counter-clockwise vertex order seen from the
outside (outward normals), which is what an RWG discretisation of a closed
PEC body expects.
"""

import numpy as np


def icosphere(subdivisions: int, radius: float):
    """Icosahedron refined ``subdivisions`` times (each triangle into four),
    vertices projected onto the sphere of the given radius.

    subdivisions=3 gives 1,280 triangles / 1,920 edges; 5 gives 20,480 / 30,720.
    Midpoints are created in a fixed order, so the output is bit-reproducible.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    for _ in range(subdivisions):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    xyz = np.array(v, dtype=np.float64) * radius
    tri = np.array(faces, dtype=np.int32)
    _orient_outward(xyz, tri)
    return xyz, tri


def _orient_outward(xyz, tri):
    """Flip triangles whose normal points towards the body centroid (in place).
    Valid for star-shaped bodies about their vertex centroid."""
    c = xyz.mean(axis=0)
    p0, p1, p2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    inward = np.einsum('ij,ij->i', n, (p0 + p1 + p2) / 3.0 - c) < 0
    tri[inward, 1], tri[inward, 2] = tri[inward, 2].copy(), tri[inward, 1].copy()


def box_surface(size, n):
    """Closed surface of an axis-aligned box ``size = (sx, sy, sz)`` centred at
    the origin, each face split into an ``n[i] x n[j]`` grid of squares, each
    square into two triangles along a fixed diagonal."""
    sx, sy, sz = size
    nx, ny, nz = n
    xs = np.linspace(-sx / 2, sx / 2, nx + 1)
    ys = np.linspace(-sy / 2, sy / 2, ny + 1)
    zs = np.linspace(-sz / 2, sz / 2, nz + 1)
    index = {}
    verts = []

    def vid(p):
        key = tuple(np.round(np.asarray(p) * 1e9).astype(np.int64))
        if key not in index:
            index[key] = len(verts)
            verts.append(p)
        return index[key]

    tris = []

    def face(u, w, fixed_axis, fixed_val):
        for i in range(len(u) - 1):
            for j in range(len(w) - 1):
                quad = []
                for (a, b) in ((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)):
                    p = [0.0, 0.0, 0.0]
                    axes = [ax for ax in range(3) if ax != fixed_axis]
                    p[axes[0]], p[axes[1]], p[fixed_axis] = u[a], w[b], fixed_val
                    quad.append(vid(tuple(p)))
                tris.append((quad[0], quad[1], quad[2]))
                tris.append((quad[0], quad[2], quad[3]))

    face(ys, zs, 0, -sx / 2), face(ys, zs, 0, sx / 2)
    face(xs, zs, 1, -sy / 2), face(xs, zs, 1, sy / 2)
    face(xs, ys, 2, -sz / 2), face(xs, ys, 2, sz / 2)
    xyz = np.array(verts, dtype=np.float64)
    tri = np.array(tris, dtype=np.int32)
    _orient_outward(xyz, tri)
    return xyz, tri


def closed_cylinder(radius, height, n_around, n_along, n_rings):
    """Closed circular cylinder along z (side wall plus two flat caps made of
    concentric rings), centred at the origin."""
    verts = []
    tris = []
    ang = 2 * np.pi * np.arange(n_around) / n_around
    zs = np.linspace(-height / 2, height / 2, n_along + 1)
    side = np.zeros((n_along + 1, n_around), dtype=np.int64)
    for i, z in enumerate(zs):
        for j, a in enumerate(ang):
            side[i, j] = len(verts)
            verts.append((radius * np.cos(a), radius * np.sin(a), z))
    for i in range(n_along):
        for j in range(n_around):
            j1 = (j + 1) % n_around
            tris.append((side[i, j], side[i, j1], side[i + 1, j1]))
            tris.append((side[i, j], side[i + 1, j1], side[i + 1, j]))
    for ring_row, z in ((0, zs[0]), (n_along, zs[-1])):
        outer = side[ring_row]
        for r in range(n_rings - 1, 0, -1):
            rr = radius * r / n_rings
            inner = []
            for a in ang:
                inner.append(len(verts))
                verts.append((rr * np.cos(a), rr * np.sin(a), z))
            for j in range(n_around):
                j1 = (j + 1) % n_around
                tris.append((outer[j], outer[j1], inner[j1]))
                tris.append((outer[j], inner[j1], inner[j]))
            outer = inner
        centre = len(verts)
        verts.append((0.0, 0.0, z))
        for j in range(n_around):
            tris.append((outer[j], outer[(j + 1) % n_around], centre))
    xyz = np.array(verts, dtype=np.float64)
    tri = np.array(tris, dtype=np.int32)
    _orient_outward(xyz, tri)
    return xyz, tri


def cube_tets(n, size=1.0):
    """Cube [-size/2, size/2]^3 split into n^3 voxels, each voxel into the 6
    tetrahedra around its main diagonal (Freudenthal subdivision; conforming
    across voxels).  Returns (xyz float64 (nv,3), tet int32 (nt,4)) with
    positive orientation."""
    g = np.linspace(-size / 2, size / 2, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for p in perms:
                    c = [0, 0, 0]
                    path = [vid(i, j, k)]
                    for ax in p:
                        c[ax] = 1
                        path.append(vid(i + c[0], j + c[1], k + c[2]))
                    tets.append(path)
    tet = np.array(tets, dtype=np.int32)
    _orient_tets(xyz, tet)
    return xyz, tet


def ball_tets(n, radius):
    """Tetrahedral mesh of a ball: the cube mesh of cube_tets(n, 2) mapped
    radially, p -> radius * p * |p|_inf / |p|_2, so that the cube surface lands
    on the sphere."""
    xyz, tet = cube_tets(n, 2.0)
    ninf = np.abs(xyz).max(axis=1)
    n2 = np.linalg.norm(xyz, axis=1)
    s = np.where(n2 > 0, ninf / np.where(n2 > 0, n2, 1.0), 0.0)
    xyz = radius * xyz * s[:, None]
    _orient_tets(xyz, tet)
    return xyz, tet


def _orient_tets(xyz, tet):
    """Swap two vertices of negatively oriented tetrahedra (in place)."""
    p = xyz[tet]
    vol = np.einsum('ij,ij->i', np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    neg = vol < 0
    tet[neg, 2], tet[neg, 3] = tet[neg, 3].copy(), tet[neg, 2].copy()


def random_permittivity(n_tet, lo, hi, seed):
    """Relative permittivity per tetrahedron, iid uniform in [lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, n_tet)


def plate(size, n):
    """Open square PEC plate [-sx/2, sx/2] x [-sy/2, sy/2] in z = 0, n = (nx, ny)
    squares, each split into two triangles along a fixed diagonal; normals +z.
    Only interior edges carry RWG unknowns (open surface)."""
    sx, sy = size
    nx, ny = n
    xs = np.linspace(-sx / 2, sx / 2, nx + 1)
    ys = np.linspace(-sy / 2, sy / 2, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)

    def vid(i, j):
        return i * (ny + 1) + j

    tris = []
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    return xyz, np.array(tris, dtype=np.int32)


def box_tets(size, n):
    """Box [-sx/2, sx/2] x [-sy/2, sy/2] x [-sz/2, sz/2] split into n = (nx, ny, nz)
    voxels of 6 tetrahedra each (the Freudenthal split of cube_tets), positive
    orientation."""
    sx, sy, sz = size
    nx, ny, nz = n
    g = [np.linspace(-s / 2, s / 2, k + 1) for s, k in ((sx, nx), (sy, ny), (sz, nz))]
    X, Y, Z = np.meshgrid(*g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                for p in perms:
                    c = [0, 0, 0]
                    path = [vid(i, j, k)]
                    for ax in p:
                        c[ax] = 1
                        path.append(vid(i + c[0], j + c[1], k + c[2]))
                    tets.append(path)
    tet = np.array(tets, dtype=np.int32)
    _orient_tets(xyz, tet)
    return xyz, tet


def shell_tets(r_in, r_out, length, n):
    """Hollow circular cylinder along z (radii r_in < r_out, length), a structured
    (n_r, n_theta, n_z) grid in (r, theta, z), periodic in theta, each cell split
    into 6 tetrahedra (Freudenthal split of the index cube, so that neighbouring
    cells share faces), positive orientation."""
    n_r, n_t, n_z = n
    rs = np.linspace(r_in, r_out, n_r + 1)
    ts = 2 * np.pi * np.arange(n_t) / n_t
    zs = np.linspace(-length / 2, length / 2, n_z + 1)

    def vid(i, j, k):
        return (i * n_t + (j % n_t)) * (n_z + 1) + k

    xyz = np.zeros(((n_r + 1) * n_t * (n_z + 1), 3))
    for i, r in enumerate(rs):
        for j, t in enumerate(ts):
            for k, z in enumerate(zs):
                xyz[vid(i, j, k)] = (r * np.cos(t), r * np.sin(t), z)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for i in range(n_r):
        for j in range(n_t):
            for k in range(n_z):
                for p in perms:
                    c = [0, 0, 0]
                    path = [vid(i, j, k)]
                    for ax in p:
                        c[ax] = 1
                        path.append(vid(i + c[0], j + c[1], k + c[2]))
                    tets.append(path)
    tet = np.array(tets, dtype=np.int32)
    _orient_tets(xyz, tet)
    return xyz, tet
