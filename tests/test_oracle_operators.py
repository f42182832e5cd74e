"""Pins of the oracle operators (Sec. 2, Sec. 3, Sec. 4) against closed forms,
invariants and the paper's convergence claims. CPU only."""

import numpy as np
import pytest
import sympy as sp

from conftest import oracle_grid
from oracle import operators as op
from oracle.grid import lonlat

# ------------------------------------------------------------- exact fields


def _heikes_exact(m, n):
    """Test functions of Sec. 2.2 (Eq. div_test) on the unit sphere, with the
    exact divergence derived symbolically from the spherical divergence
    formula (independent of the printed components, reading: the i-component
    carries sin(lambda), as alpha = sin(lambda) implies)."""
    lam, phi = sp.symbols("lam phi", real=True)
    alpha = sp.sin(lam)
    beta = sp.cos(m * lam) * sp.cos(n * phi) ** 4
    gl = sp.diff(beta, lam) / sp.cos(phi)     # lambda component of grad beta
    gp = sp.diff(beta, phi)
    vl, vp = alpha * gl, alpha * gp
    div = (sp.diff(vl, lam) + sp.diff(vp * sp.cos(phi), phi)) / sp.cos(phi)
    f = lambda e: sp.lambdify((lam, phi), sp.simplify(e), "numpy")
    return f(beta), f(gl), f(gp), f(vl), f(vp), f(div)


def _unit_vectors(P):
    lon, lat = lonlat(P)
    elon = np.stack([-np.sin(lon), np.cos(lon), 0 * lon], 1)
    elat = np.stack([-np.sin(lat) * np.cos(lon), -np.sin(lat) * np.sin(lon), np.cos(lat)], 1)
    return lon, lat, elon, elat


def _heikes_errors(G, m, n):
    beta, gl, gp, vl, vp, div = _heikes_exact(m, n)
    lon, lat, elon, elat = _unit_vectors(G.points)
    v = vl(lon, lat)[:, None] * elon + vp(lon, lat)[:, None] * elat
    e = op.div_h(G, v) - div(lon, lat)
    w = G.area / G.area.sum()
    grad_ex = gl(lon, lat)[:, None] * elon + gp(lon, lat)[:, None] * elat
    eg = np.linalg.norm(op.grad_h(G, beta(lon, lat)) - grad_ex, axis=1)
    return (np.sqrt(np.sum(w * e ** 2)), np.abs(e).max(),
            np.sqrt(np.sum(w * eg ** 2)), eg.max())


# ------------------------------------------------------------- pins


def test_gradient_of_constant_vanishes():
    """Sec. 2.1: the curvature term of Eq. grad makes grad(const) zero."""
    for modified in (False, True):
        G = oracle_grid(3, modified=modified)
        g = op.grad_h(G, np.full(G.ncol, 7.0e4), project=False)
        assert np.max(np.abs(g)) < 1e-14 * 7.0e4 * 2 ** 3


def test_discrete_gauss_conservation():
    """Flux form: sum_cells A_c div(Phi) = 0 for any Phi (exact telescoping)."""
    G = oracle_grid(3)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((G.ncol, 4, 3))
    s = np.einsum("i,ik->k", G.area, op.div_h(G, v))
    assert np.max(np.abs(s)) < 1e-13 * np.abs(v).max()
    lap = np.einsum("i,ik->k", G.area, op.laplacian(G, v[..., 0]))
    assert np.max(np.abs(lap)) < 1e-12 * np.abs(v).max()


def test_heikes_second_order_modified_grid():
    """Sec. 2.2: the l2 error of the divergence and gradient of the Heikes test
    functions converges at second order on the modified grid, and the
    modified grid beats the standard one."""
    errs = {g: _heikes_errors(oracle_grid(g), 1, 1) for g in (2, 3, 4)}
    std4 = _heikes_errors(oracle_grid(4, modified=False), 1, 1)
    slope_div = np.log2(errs[3][0] / errs[4][0])
    slope_grad = np.log2(errs[3][2] / errs[4][2])
    assert 1.8 < slope_div < 2.2, slope_div
    assert 1.8 < slope_grad < 2.2, slope_grad
    assert errs[4][0] < std4[0] and errs[4][1] < std4[1]
    assert errs[4][2] < std4[2] and errs[4][3] < std4[3]
    e33 = _heikes_errors(oracle_grid(4), 3, 3)
    s33 = _heikes_errors(oracle_grid(4, modified=False), 3, 3)
    assert e33[0] < s33[0]


def _away_from_pentagons(G, rings=2):
    near = set(np.where(G.nn == 5)[0].tolist())
    for _ in range(rings):
        for i in list(near):
            near.update(G.nbr[i, :G.nn[i]].tolist())
    mask = np.ones(G.ncol, bool)
    mask[list(near)] = False
    return mask


@pytest.mark.parametrize("ell, field", [(1, lambda P: P[:, 2]), (2, lambda P: P[:, 0] * P[:, 1]),
                                        (3, lambda P: P[:, 0] * P[:, 1] * P[:, 2])])
def test_laplacian_spherical_harmonics(ell, field):
    """Sec. 4 Laplacian: lap Y_l = -l(l+1) Y_l on the unit sphere. Away from
    the twelve pentagons the error falls at second order; at a pentagon the
    five triangle gradients cannot cancel their first-order errors in pairs,
    so the error there stays bounded but does not fall."""
    errs, maxes = [], []
    for g in (3, 4):
        G = oracle_grid(g)
        s = field(G.points)
        e = op.laplacian(G, s) + ell * (ell + 1) * s
        m = _away_from_pentagons(G)
        errs.append(np.sqrt(np.sum((G.area * e ** 2)[m]) / np.sum(G.area[m])))
        maxes.append(np.abs(e).max())
    assert np.log2(errs[0] / errs[1]) > 1.8
    assert errs[1] < 2e-3 * ell * (ell + 1)
    assert maxes[1] < 0.1 * ell * (ell + 1)


def test_lagrange_linear_interpolation_exact():
    vg = op.VerticalGrid(7, 1.0e4, 6.4e6)
    f = 3.0 + 2.0e-3 * vg.zc
    fi = op.interp_to_interfaces(vg, f)
    assert np.allclose(fi[1:-1], 3.0 + 2.0e-3 * vg.zi[1:-1], rtol=0, atol=1e-13)
    g = -1.0 + 5.0e-4 * vg.zi
    assert np.allclose(op.interp_to_centres(vg, g), -1.0 + 5.0e-4 * vg.zc, rtol=0, atol=1e-13)


def test_deep_vertical_divergence():
    """Sec. 3, 3-D split: r^-2 d(r^2 W)/dr vanishes for W ~ r^-2 (exact
    telescoping) and is 3 + dz^2/(4 r_c^2) for W = r (midpoint rule)."""
    vg = op.VerticalGrid(10, 3.0e4, 6.4e6)
    W = 1.0 / vg.ri ** 2
    assert np.max(np.abs(op.div_v(vg, W))) < 1e-28
    d = op.div_v(vg, vg.ri.copy())
    assert np.allclose(d, 3.0 + vg.dz ** 2 / (4 * vg.rc ** 2), rtol=1e-12)


def test_projection():
    rng = np.random.default_rng(1)
    r = rng.standard_normal((5, 3))
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    v = rng.standard_normal((5, 2, 3))
    vh = op.project_h(r, v)
    assert np.max(np.abs(np.sum(vh * r[:, None, :], -1))) < 1e-15
    back = vh + op.radial(r, v)[..., None] * r[:, None, :]
    assert np.allclose(back, v, atol=1e-15)
