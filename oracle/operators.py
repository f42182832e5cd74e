"""Oracle discrete operators of Sec. 2 and Sec. 3-4, float64, unit sphere.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Horizontal operators act on arrays whose first axis is the cell index; any
further axes (levels, vector components) broadcast. They are written on the
unit sphere; at radius r a horizontal divergence or gradient is divided by r
and the Laplacian by r^2 (deep atmosphere, Sec. 3: the control volume at
radius r has area A_c r^2 and edges l_k r).

Readings:

* Corner values are defined once per triangle (Eq. int_grid is symmetric in
  the triangle's three vertices), so both cells that share an edge see the
  same corner values and the flux of Eq. flx_div is exactly antisymmetric.
* The horizontal gradient is Eq. grad followed by the horizontal projection
  of Eq. proj_h, read as Phi - (Phi . r) r (the printed Phi - Phi . r is
  garbled).
* The Laplacian of Sec. 4: on every triangle (P_0, P_k, P_k+1) Eq. grad is
  applied with the triangle as control volume (its edges are the arcs between
  the P's, the edge value is the mean of the two end values, the centre value
  is the corner value of Eq. int_grid), which places a gradient vector at the
  corner C_k; Eq. div_gauss applied to those corner vectors gives the
  Laplacian at P_0.
* Vertical interpolation is the Lagrange polynomial of Sec. 2.1, k = 1
  (linear in altitude) by default, from centres to interfaces and back.
* Reading L-1 (Sec. 2.1 leaves the nodes of a k > 1 polynomial unstated):
  the k + 1 consecutive nodes nearest the target, the lower one first where
  two are equally near (even k), shifted inward at the bottom and the top.
"""

import numpy as np


def _bc(geom, like):
    """Reshape per-cell (or per-face) geometry ``geom`` with shape (M, ...) so
    that it broadcasts against ``like`` with shape (M, *extra)."""
    extra = like.ndim - 1
    return geom.reshape(geom.shape[:1] + (1,) * extra)


def corner_values(grid, phi):
    """Eq. int_grid: value at every triangle corner C from the triangle's
    three vertices, weighted by the areas of the opposite sub-triangles."""
    out = 0.0
    for v in range(3):
        w = grid.tri_w[:, v]
        x = phi[grid.faces[:, v]]
        out = out + _bc(w, x) * x
    return out


def div_corner_vectors(grid, cvec):
    """Eqs. flx_div and div_gauss for vectors given at the corners:
    (1/A_c) sum_k l_k (Phi*_k + Phi*_k+1)/2 . n_k. ``cvec`` has shape
    (F, ..., 3); the result has shape (N, ...)."""
    N = grid.ncol
    out = 0.0
    idx = np.arange(N)
    for k in range(6):
        valid = (k < grid.nn).astype(float)
        kn = np.where(k + 1 < grid.nn, k + 1, 0)
        fk = grid.ring_face[idx, np.where(k < grid.nn, k, 0)]
        fk1 = grid.ring_face[idx, kn]
        mean = 0.5 * (cvec[fk] + cvec[fk1])                  # (N, ..., 3)
        n = grid.edge_n[:, k].reshape((N,) + (1,) * (cvec.ndim - 2) + (3,))
        flux = np.sum(mean * n, axis=-1)                     # (N, ...)
        out = out + _bc(valid * grid.edge_l[:, k], flux) * flux
    return out / _bc(grid.area, out)


def div_h(grid, vec):
    """Horizontal divergence (Eq. div_gauss) of cell-centred 3-D vectors."""
    return div_corner_vectors(grid, corner_values(grid, vec))


def project_h(rhat, vec):
    """Eq. proj_h read as Phi - (Phi . r) r; ``rhat`` (N, 3)."""
    r = rhat.reshape((rhat.shape[0],) + (1,) * (vec.ndim - 2) + (3,))
    return vec - np.sum(vec * r, axis=-1, keepdims=True) * r


def radial(rhat, vec):
    """Eq. proj_r: Phi . r."""
    r = rhat.reshape((rhat.shape[0],) + (1,) * (vec.ndim - 2) + (3,))
    return np.sum(vec * r, axis=-1)


def grad_h(grid, s, project=True):
    """Eq. grad: (1/A_c) sum_k l_k (s*_k + s*_k+1)/2 n_k - (s_0/A_c) sum_k l_k n_k,
    then the horizontal projection. ``s`` (N, ...) -> (N, ..., 3)."""
    N = grid.ncol
    sc = corner_values(grid, s)
    idx = np.arange(N)
    acc = 0.0
    lsum = np.zeros((N, 3))
    for k in range(6):
        valid = (k < grid.nn).astype(float)
        kn = np.where(k + 1 < grid.nn, k + 1, 0)
        fk = grid.ring_face[idx, np.where(k < grid.nn, k, 0)]
        fk1 = grid.ring_face[idx, kn]
        ln = (valid * grid.edge_l[:, k])[:, None] * grid.edge_n[:, k]      # (N, 3)
        mean = 0.5 * (sc[fk] + sc[fk1])                                    # (N, ...)
        acc = acc + mean[..., None] * ln.reshape((N,) + (1,) * (s.ndim - 1) + (3,))
        lsum += ln
    acc = acc - s[..., None] * lsum.reshape((N,) + (1,) * (s.ndim - 1) + (3,))
    out = acc / grid.area.reshape((N,) + (1,) * s.ndim)
    return project_h(grid.points, out) if project else out


def triangle_gradients(grid, s):
    """Sec. 4: Eq. grad applied to every primary triangle; returns the
    gradient vector at each corner C, shape (F, ..., 3)."""
    F = len(grid.faces)
    sc = corner_values(grid, s)
    acc = 0.0
    lsum = np.zeros((F, 3))
    for v in range(3):
        u = grid.faces[:, v]
        w = grid.faces[:, (v + 1) % 3]
        ln = grid.tri_edge_l[:, v][:, None] * grid.tri_edge_n[:, v]
        mean = 0.5 * (s[u] + s[w])
        acc = acc + mean[..., None] * ln.reshape((F,) + (1,) * (s.ndim - 1) + (3,))
        lsum += ln
    acc = acc - sc[..., None] * lsum.reshape((F,) + (1,) * (s.ndim - 1) + (3,))
    return acc / grid.tri_area.reshape((F,) + (1,) * s.ndim)


def laplacian(grid, s):
    """Sec. 4: horizontal Laplacian = Eq. div_gauss of the triangle gradients
    placed at the corners. ``s`` (N, ...) -> (N, ...)."""
    return div_corner_vectors(grid, triangle_gradients(grid, s))


def vector_laplacian(grid, vec):
    """Component-wise Cartesian Laplacian (Sec. 4: operators formulated in
    Cartesian coordinates). ``vec`` (N, ..., 3)."""
    return np.stack([laplacian(grid, vec[..., j]) for j in range(3)], axis=-1)


# ---------------------------------------------------------------- vertical

class VerticalGrid:
    """Layers of the deep atmosphere (Sec. 2.1, Sec. 3).

    Reading: the paper does not give the layer spacing; we take uniform
    layers, interfaces z_i = i dz (i = 0..nv) and centres z_k = (k + 1/2) dz.
    r = radius + z. The cell volume is A_c r_k^2 (z_k+1/2 - z_k-1/2).
    shallow: the shallow-atmosphere approximation of Sec. 3 (1/r replaced by
    1/A, A the planet radius): r = A at every centre and interface, the
    heights z unchanged (reading S-1)."""

    def __init__(self, nv, z_top, radius, shallow=False):
        self.nv = nv
        self.radius = radius
        self.shallow = shallow
        self.zi = np.linspace(0.0, z_top, nv + 1)
        self.zc = 0.5 * (self.zi[:-1] + self.zi[1:])
        self.dz = np.diff(self.zi)
        self.rc = radius + (0.0 if shallow else 1.0) * self.zc
        self.ri = radius + (0.0 if shallow else 1.0) * self.zi


def lagrange_weights(nodes, zh):
    """Sec. 2.1: the weights L_j(z_h) = prod_{i != j} (z_h - z_i) / (z_j - z_i)
    of the Lagrange polynomial through ``nodes`` (k + 1 altitudes), so that
    Phi(z_h) = sum_j Phi_j L_j(z_h)."""
    w = np.ones(len(nodes))
    for j, zj in enumerate(nodes):
        for i, zi in enumerate(nodes):
            if i != j:
                w[j] *= (zh - zi) / (zj - zi)
    return w


def stencil_start(target, k, n):
    """First of the k + 1 consecutive nodes used for the target position
    (reading L-1): the nodes nearest the target, target - ceil((k + 1) / 2)
    up, shifted inward where they would leave the n nodes. ``target`` is the
    index of the first node above the target position."""
    return min(max(target - (k + 2) // 2, 0), n - k - 1)


def interp_to_interfaces(vg, x, order=1):
    """Lagrange interpolation of order k = ``order`` (Sec. 2.1) from centres
    to the interior interfaces: x (..., nv) -> (..., nv+1) with the two
    boundary interfaces left at 0. k = 1 is linear in altitude between the
    two centres around the interface; k > 1 takes the k + 1 centres of
    stencil_start."""
    out = np.zeros(x.shape[:-1] + (vg.nv + 1,))
    if order == 1:
        z0, z1 = vg.zc[:-1], vg.zc[1:]
        zh = vg.zi[1:-1]
        out[..., 1:-1] = x[..., :-1] * (zh - z1) / (z0 - z1) + x[..., 1:] * (zh - z0) / (z1 - z0)
        return out
    if vg.nv < order + 1:
        raise ValueError("fewer centres than the interpolation order needs")
    for i in range(1, vg.nv):
        j0 = stencil_start(i, order, vg.nv)
        w = lagrange_weights(vg.zc[j0:j0 + order + 1], vg.zi[i])
        out[..., i] = sum(w[j] * x[..., j0 + j] for j in range(order + 1))
    return out


def interp_to_centres(vg, xi, order=1):
    """Lagrange interpolation of order k = ``order`` from interfaces to
    centres: xi (..., nv+1) -> (..., nv). k = 1 is linear between the two
    interfaces of the layer; k > 1 takes the k + 1 interfaces of
    stencil_start (the boundary interfaces included)."""
    if order == 1:
        z0, z1 = vg.zi[:-1], vg.zi[1:]
        zh = vg.zc
        return xi[..., :-1] * (zh - z1) / (z0 - z1) + xi[..., 1:] * (zh - z0) / (z1 - z0)
    if vg.nv + 1 < order + 1:
        raise ValueError("fewer interfaces than the interpolation order needs")
    out = np.zeros(xi.shape[:-1] + (vg.nv,))
    for c in range(vg.nv):
        j0 = stencil_start(c + 1, order, vg.nv + 1)
        w = lagrange_weights(vg.zi[j0:j0 + order + 1], vg.zc[c])
        out[..., c] = sum(w[j] * xi[..., j0 + j] for j in range(order + 1))
    return out


def ddz_at_interfaces(vg, x):
    """d/dr at the interior interfaces from centre values; 0 at the boundaries."""
    out = np.zeros(x.shape[:-1] + (vg.nv + 1,))
    out[..., 1:-1] = (x[..., 1:] - x[..., :-1]) / (vg.zc[1:] - vg.zc[:-1])
    return out


def div_v(vg, wi):
    """Radial part of the deep divergence (Sec. 3, 3-D operator split):
    r^-2 d(r^2 W)/dr at the centres from interface values wi (..., nv+1)."""
    f = vg.ri ** 2 * wi
    return (f[..., 1:] - f[..., :-1]) / (vg.rc ** 2 * vg.dz)


def div_h_levels(grid, vg, vec, at_interfaces=False):
    """Horizontal divergence at every level: vec (N, L, 3); divided by r."""
    r = vg.ri if at_interfaces else vg.rc
    return div_h(grid, vec) / r[None, :]


def grad_h_levels(grid, vg, s, at_interfaces=False):
    r = vg.ri if at_interfaces else vg.rc
    return grad_h(grid, s) / r[None, :, None]


def lap_levels(grid, vg, s, at_interfaces=False):
    r = vg.ri if at_interfaces else vg.rc
    return laplacian(grid, s) / (r[None, :] ** 2)


def vlap_levels(grid, vg, vec):
    return vector_laplacian(grid, vec) / (vg.rc[None, :, None] ** 2)
