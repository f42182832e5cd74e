"""Oracle grid: the icosahedral grid of Sec. 2, on the unit sphere, in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The construction follows Sec. 2 in the paper's order:

1. Standard icosahedral grid (Sec. 2.1): an icosahedron with two vertices at
   the poles, refined ``glevel`` times by bisecting every triangle edge and
   projecting the midpoint onto the sphere (Fig. icogrid).
2. Spring dynamics (Sec. 2.2, Eqs. spring_force, spr_vel, dbar), with the
   twelve pentagon centres held fixed.
3. Centroid relocation (Sec. 2.2): the control-volume vertices C_k are moved
   to the centroids of the triangles, then, with the C_k held fixed, every
   point P is moved to the centroid of its control volume.
4. Metric terms (Sec. 2.1): arc lengths l_k, outward unit normals n_k,
   control-volume areas A_c and the sub-triangle areas A_1, A_2, A_3 of
   Eq. int_grid.

This module uses a generic triangle list (faces) with creation-order
numbering; it shares nothing with the CUDA path's grid builder, which uses its
own numbering. Tests relate the two by matching point coordinates.

Readings of silent or garbled passages:

* Icosahedron orientation: north pole, five vertices at latitude +atan(1/2)
  and longitudes 0, 72, ... deg, five at latitude -atan(1/2) and longitudes
  36, 108, ... deg, south pole.
* Spring dynamics: the paper gives Eq. spring_force but not the integrator or
  the spring constant. We take k = 1 and the semi-implicit Euler step
  v <- v + dt (F - alpha v); P <- normalize(P + dt v); v <- v - (v.P) P.
  d_i is the great-circle arc from P_0 to P_i and e_i the unit tangent at P_0
  pointing to P_i. The stop rule "no point moves more than 1e-5" is read as
  max |v| < 1e-5 (movement per unit of the nondimensional time).
* The centroid formula of Sec. 2.2 prints atan(|r_i . r_i+1| / |r_i x r_i+1|),
  which is the complement of the arc angle. We use the arc angle
  theta_i = atan2(|r_i x r_i+1|, r_i . r_i+1); then
  sum_i theta_i (r_i x r_i+1)/|r_i x r_i+1| is the first moment of the
  spherical polygon, and its direction is the centroid (the 1/(2 pi) factor
  drops out after normalisation).
* Spherical triangle areas use the Van Oosterom-Strackee formula
  tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a).
* The outward normal n_k of the arc C_k -> C_k+1 is the unit normal of the
  great-circle plane through C_k and C_k+1, signed so that n_k . P_0 < 0. It
  is tangent to the sphere and perpendicular to the arc along the whole arc.
"""

from dataclasses import dataclass

import numpy as np


def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def arc(a, b):
    """Great-circle arc (radians) between unit vectors a and b."""
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def spherical_triangle_area(a, b, c):
    """Area of the spherical triangle (a, b, c) on the unit sphere
    (Van Oosterom-Strackee; orientation-free)."""
    num = np.abs(np.sum(a * np.cross(b, c), axis=-1))
    den = 1.0 + np.sum(a * b, axis=-1) + np.sum(b * c, axis=-1) + np.sum(c * a, axis=-1)
    return 2.0 * np.arctan2(num, den)


def spherical_centroid(verts):
    """Centroid of the spherical polygon whose vertices ``verts[..., i, :]``
    are listed counter-clockwise (Sec. 2.2, centroid equation, with the arc
    angle reading stated in the module docstring)."""
    r0 = verts
    r1 = np.roll(verts, -1, axis=-2)
    cr = np.cross(r0, r1)
    s = np.linalg.norm(cr, axis=-1, keepdims=True)
    theta = np.arctan2(s, np.sum(r0 * r1, axis=-1, keepdims=True))
    m = np.sum(theta * cr / s, axis=-2)
    return _normalize(m)


def icosahedron():
    """The 12 vertices and 20 faces of the icosahedron with two vertices at
    the poles (Sec. 2.1). Faces are counter-clockwise seen from outside."""
    lat = np.arctan(0.5)
    pts = [np.array([0.0, 0.0, 1.0])]
    for k in range(5):
        lon = 2.0 * np.pi * k / 5.0
        pts.append(np.array([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)]))
    for k in range(5):
        lon = 2.0 * np.pi * k / 5.0 + np.pi / 5.0
        pts.append(np.array([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), -np.sin(lat)]))
    pts.append(np.array([0.0, 0.0, -1.0]))
    N, S = 0, 11
    faces = []
    for k in range(5):
        u0, u1 = 1 + k, 1 + (k + 1) % 5
        l0, l1 = 6 + k, 6 + (k + 1) % 5
        faces += [(N, u0, u1), (u0, l0, u1), (l0, l1, u1), (S, l1, l0)]
    pts = np.array(pts)
    faces = np.array(faces, dtype=np.int64)
    # orient every face counter-clockwise seen from outside
    a, b, c = pts[faces[:, 0]], pts[faces[:, 1]], pts[faces[:, 2]]
    flip = np.sum(np.cross(b - a, c - a) * (a + b + c), axis=1) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    return pts, faces


def bisect(points, faces):
    """One refinement of Fig. icogrid: every edge is bisected, the midpoint is
    projected onto the sphere, and each triangle becomes four."""
    F = len(faces)
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    es = np.sort(e, axis=1)
    uniq, inv = np.unique(es, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    mids = _normalize(points[uniq[:, 0]] + points[uniq[:, 1]])
    mid_id = len(points) + inv
    ab, bc, ca = mid_id[:F], mid_id[F:2 * F], mid_id[2 * F:]
    a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
    new = np.concatenate([
        np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
        np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)])
    return np.concatenate([points, mids]), new


def neighbour_rings(npts, faces):
    """Counter-clockwise ring of neighbours and of incident faces for every
    point. Returns ``nbr`` (N, 6), ``ring_face`` (N, 6) padded with -1 for the
    pentagons and ``nn`` (N,). ``ring_face[i, k]`` is the face
    (i, nbr[i, k], nbr[i, k+1])."""
    succ = [dict() for _ in range(npts)]
    face_of = [dict() for _ in range(npts)]
    for f, (a, b, c) in enumerate(faces):
        for v, x, y in ((a, b, c), (b, c, a), (c, a, b)):
            succ[v][x] = y
            face_of[v][x] = f
    nbr = -np.ones((npts, 6), dtype=np.int64)
    ring_face = -np.ones((npts, 6), dtype=np.int64)
    nn = np.zeros(npts, dtype=np.int64)
    for v in range(npts):
        start = min(succ[v])
        ring = [start]
        while True:
            nxt = succ[v][ring[-1]]
            if nxt == start:
                break
            ring.append(nxt)
        m = len(ring)
        assert m == len(succ[v]) and m in (5, 6)
        nn[v] = m
        nbr[v, :m] = ring
        ring_face[v, :m] = [face_of[v][x] for x in ring]
    return nbr, ring_face, nn


def natural_spring_length(glevel, beta, radius=1.0):
    """Eq. dbar: natural spring length beta * 2 pi A / (10 * 2^(glevel-1))."""
    return beta * 2.0 * np.pi * radius / (10.0 * 2.0 ** (glevel - 1))


def spring_dynamics(points, nbr, nn, glevel, beta=1.15, alpha=1.0, k=1.0, dt=0.01,
                    tol=1e-5, max_iter=100000):
    """Eqs. spring_force and spr_vel integrated on the unit sphere.

    Every point is tied to its neighbours by springs of natural length
    Eq. dbar; the twelve pentagon centres stay fixed. The loop stops when no
    point moved more than ``tol`` in the last step (tol > 0) or after
    ``max_iter`` steps. Returns (points, iterations, converged).

    Reading of the stopping rule: the paper stops when no point moves more
    than 1e-5. Taken per step of dt = 0.01 from rest, that holds after the
    first step (the first displacement is dt^2 |F|), so we read the rule per
    unit of the nondimensional time of Eq. spr_vel: stop when every
    |v| = |dP/dt| < tol."""
    P = points.copy()
    v = np.zeros_like(P)
    valid = nbr >= 0
    nb = np.where(valid, nbr, np.arange(len(P))[:, None])
    fixed = nn == 5
    dbar = natural_spring_length(glevel, beta)
    it = 0
    converged = False
    while it < max_iter:
        Q = P[nb]                                            # (N, 6, 3)
        dot = np.sum(P[:, None, :] * Q, axis=-1)
        d = np.arctan2(np.linalg.norm(np.cross(P[:, None, :], Q), axis=-1), dot)
        t = Q - dot[..., None] * P[:, None, :]
        tn = np.linalg.norm(t, axis=-1, keepdims=True)
        e = np.where(valid[..., None], t / np.where(tn > 0, tn, 1.0), 0.0)
        force = np.sum(np.where(valid, k * (d - dbar), 0.0)[..., None] * e, axis=1)
        force[fixed] = 0.0
        v = v + dt * (force - alpha * v)
        v[fixed] = 0.0

        Pn = _normalize(P + dt * v)
        Pn[fixed] = P[fixed]
        v = v - np.sum(v * Pn, axis=1, keepdims=True) * Pn
        speed = np.max(np.linalg.norm(v, axis=1))
        P = Pn
        it += 1
        if tol > 0 and speed < tol:
            converged = True
            break
    return P, it, converged


@dataclass
class Grid:
    glevel: int
    points: np.ndarray      # (N, 3) cell centres P
    faces: np.ndarray       # (F, 3) triangles, counter-clockwise
    nbr: np.ndarray         # (N, 6) neighbours, counter-clockwise, -1 padded
    nn: np.ndarray          # (N,) 5 or 6
    ring_face: np.ndarray   # (N, 6) faces around each cell (C_k), -1 padded
    corners: np.ndarray     # (F, 3) control-volume vertices C (triangle centroids)
    tri_w: np.ndarray       # (F, 3) Eq. int_grid weights of the face's 3 vertices
    edge_l: np.ndarray      # (N, 6) arc C_k -> C_k+1
    edge_n: np.ndarray      # (N, 6, 3) outward unit normal of that arc
    area: np.ndarray        # (N,) control-volume area A_c
    tri_area: np.ndarray    # (F,) spherical area of the triangle
    tri_edge_l: np.ndarray  # (F, 3) arc of triangle edge (v, v+1)
    tri_edge_n: np.ndarray  # (F, 3, 3) outward unit normal of triangle edge (v, v+1)
    spring_iters: int = 0
    spring_converged: bool = False

    @property
    def ncol(self):
        return len(self.points)


def build_grid(glevel, modified=True, beta=1.15, alpha=1.0, k=1.0, dt=0.01, tol=1e-5,
               max_iter=100000):
    """Build the standard (``modified=False``) or the modified grid of Sec. 2."""
    pts, faces = icosahedron()
    for _ in range(glevel):
        pts, faces = bisect(pts, faces)
    nbr, ring_face, nn = neighbour_rings(len(pts), faces)
    iters, conv = 0, False
    if modified and glevel > 0:
        pts, iters, conv = spring_dynamics(pts, nbr, nn, glevel, beta, alpha, k, dt, tol, max_iter)
    # control-volume vertices: centroids of the triangles
    corners = spherical_centroid(pts[faces])
    if modified:
        # move every P to the centroid of its control volume, C_k fixed
        newp = np.empty_like(pts)
        for m in (5, 6):
            sel = nn == m
            newp[sel] = spherical_centroid(corners[ring_face[sel, :m]])
        pts = newp
    return finish_metrics(glevel, pts, faces, nbr, nn, ring_face, corners, iters, conv)


def finish_metrics(glevel, pts, faces, nbr, nn, ring_face, corners, iters=0, conv=False):
    """Metric terms of Sec. 2.1 for final centres ``pts`` and fixed corners."""
    N = len(pts)
    a, b, c = pts[faces[:, 0]], pts[faces[:, 1]], pts[faces[:, 2]]
    C = corners
    # Eq. int_grid: the weight of each vertex is the area of the sub-triangle
    # opposite to it (A_2 for P_0, A_3 for P_k, A_1 for P_k+1)
    wa = spherical_triangle_area(b, c, C)
    wb = spherical_triangle_area(a, c, C)
    wc = spherical_triangle_area(a, b, C)
    tri_w = np.stack([wa, wb, wc], 1) / (wa + wb + wc)[:, None]

    edge_l = np.zeros((N, 6))
    edge_n = np.zeros((N, 6, 3))
    area = np.zeros(N)
    for kk in range(6):
        valid = kk < nn
        kn = np.where(kk + 1 < nn, kk + 1, 0)
        ck = C[np.where(valid, ring_face[:, kk], 0)]
        ck1 = C[ring_face[np.arange(N), np.where(valid, kn, 0)]]
        cr = np.cross(ck, ck1)
        crn = np.linalg.norm(cr, axis=1, keepdims=True)
        n = cr / np.where(crn > 0, crn, 1.0)
        sgn = np.where(np.sum(n * pts, axis=1) > 0, -1.0, 1.0)
        edge_n[:, kk] = np.where(valid[:, None], sgn[:, None] * n, 0.0)
        edge_l[:, kk] = np.where(valid, arc(ck, ck1), 0.0)
        area += np.where(valid, spherical_triangle_area(pts, ck, ck1), 0.0)

    tri_area = spherical_triangle_area(a, b, c)
    tri_edge_l = np.zeros((len(faces), 3))
    tri_edge_n = np.zeros((len(faces), 3, 3))
    verts = [a, b, c]
    for v in range(3):
        u, w, opp = verts[v], verts[(v + 1) % 3], verts[(v + 2) % 3]
        n = _normalize(np.cross(u, w))
        sgn = np.where(np.sum(n * opp, axis=1) > 0, -1.0, 1.0)
        tri_edge_n[:, v] = sgn[:, None] * n
        tri_edge_l[:, v] = arc(u, w)
    return Grid(glevel, pts, faces, nbr, nn, ring_face, C, tri_w, edge_l, edge_n, area,
                tri_area, tri_edge_l, tri_edge_n, iters, conv)


def mean_resolution(glevel, radius):
    """Eq. grid_qts: (N_vertices, d_bar, theta_bar)."""
    nvert = 2 + 10 * 2 ** (2 * glevel)
    dbar = np.sqrt(2.0 * np.pi / 5.0) * radius / 2.0 ** glevel
    thbar = np.sqrt(2.0 * np.pi / 5.0) / 2.0 ** glevel
    return nvert, dbar, thbar


def lonlat(points):
    """Longitude and latitude (radians) of unit vectors."""
    lon = np.arctan2(points[..., 1], points[..., 0])
    lat = np.arcsin(np.clip(points[..., 2], -1.0, 1.0))
    return lon, lat
