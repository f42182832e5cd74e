"""Pins of the oracle's vertical Lagrange interpolation of order k (Sec. 2.1)
and of the model that uses it in its explicit terms (reading L-2). CPU only."""

import numpy as np
import pytest

from conftest import oracle_grid
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls


def test_lagrange_weights_are_the_cardinal_polynomials():
    """L_j(z_i) = delta_ij at the nodes, and the weights sum to 1 anywhere
    (a constant is reproduced)."""
    nodes = np.array([0.0, 0.7, 2.1, 3.0])
    for i, zi in enumerate(nodes):
        assert np.allclose(op.lagrange_weights(nodes, zi), np.eye(4)[i], atol=1e-15)
    for zh in (-0.5, 1.3, 2.9, 4.0):
        assert abs(op.lagrange_weights(nodes, zh).sum() - 1.0) < 1e-13


def test_order_one_is_the_linear_interpolation():
    """The k = 1 path (two nodes around the target) equals the Lagrange
    polynomial through those two nodes written out generally."""
    vg = op.VerticalGrid(7, 1.0e4, 6.4e6)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 7))
    xi = op.interp_to_interfaces(vg, x, 1)
    for i in range(1, 7):
        w = op.lagrange_weights(vg.zc[i - 1:i + 1], vg.zi[i])
        assert np.allclose(xi[:, i], w[0] * x[:, i - 1] + w[1] * x[:, i], rtol=0, atol=1e-14)
    y = rng.standard_normal((3, 8))
    yc = op.interp_to_centres(vg, y, 1)
    for c in range(7):
        w = op.lagrange_weights(vg.zi[c:c + 2], vg.zc[c])
        assert np.allclose(yc[:, c], w[0] * y[:, c] + w[1] * y[:, c + 1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("nv", [5, 9])
def test_exact_on_polynomials_of_degree_k(k, nv):
    """A polynomial of degree <= k in the altitude is interpolated exactly at
    every interior interface and every centre, including where the stencil
    is shifted at the bottom and the top; degree k + 1 is not."""
    vg = op.VerticalGrid(nv, 2.0e4, 6.4e6)
    s = lambda z: z / 2.0e4
    for deg in range(k + 2):
        p = lambda z: (s(z) + 0.3) ** deg
        ei = np.abs(op.interp_to_interfaces(vg, p(vg.zc), k)[1:-1] - p(vg.zi[1:-1])).max()
        ec = np.abs(op.interp_to_centres(vg, p(vg.zi), k) - p(vg.zc)).max()
        if deg <= k:
            assert ei < 1e-13 and ec < 1e-13, (deg, ei, ec)
        else:
            assert ei > 1e-6 and ec > 1e-6, (deg, ei, ec)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_convergence_order_k_plus_one(k):
    """The interpolation error of a smooth profile falls as dz^(k+1)."""
    errs = []
    for nv in (16, 32, 64):
        vg = op.VerticalGrid(nv, 3.0e4, 6.4e6)
        f = lambda z: np.sin(2.3 * z / 3.0e4 + 0.4)
        errs.append(np.abs(op.interp_to_interfaces(vg, f(vg.zc), k)[1:-1] - f(vg.zi[1:-1])).max())
    rates = [np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])]
    assert all(k + 1 - 0.3 < r < k + 1 + 0.5 for r in rates), rates


def _model(vorder, glevel=2, nv=8, hyper=True):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    return dc.Model(oracle_grid(glevel, max_iter=10, tol=0.0), op.VerticalGrid(nv, 2.0e4, P.radius), pl,
                    vorder=vorder, hyperdiffusion=hyper)


def test_third_order_model_keeps_rest_mass_and_uniform_theta():
    """Reading L-2 keeps k = 1 in every term of the vertical system: with
    vorder = 3 a resting isothermal atmosphere in discrete balance stays at
    rest, the mass is conserved to rounding with motion, and a uniform theta
    stays uniform (diffusion off)."""
    m = _model(3)
    X = dc.initial_state(m, 280.0, 1.0e5)
    Y = dc.run(m, X, 5, 6, 1200.0)
    assert np.abs(Y.M / Y.rho[..., None]).max() < 1e-8 and np.abs(Y.W).max() < 1e-8
    rng = np.random.default_rng(2)
    X.M[:] = op.project_h(m.rhat, rng.standard_normal(X.M.shape)) * X.rho[..., None]
    X.W[:, 1:-1] = 0.01 * rng.standard_normal((X.W.shape[0], m.vg.nv - 1))
    from oracle import diagnostics as dg
    m0 = dg.diagnostics(m, X)["mass"]
    Z = dc.run(m, X, 3, 6, 1200.0)
    assert abs(dg.diagnostics(m, Z)["mass"] - m0) / m0 < 1e-13
    m2 = _model(3, hyper=False)
    X2 = dc.initial_state(m2, 280.0, 1.0e5)
    X2.M[:] = X.M
    X2.W[:] = X.W
    theta0 = X2.Th / X2.rho
    assert np.ptp(theta0) > 1.0                     # not uniform yet: isothermal, not isentropic
    # a uniform theta: rho theta proportional to rho
    X2.Th[:] = 300.0 * X2.rho
    Z2 = dc.run(m2, X2, 2, 6, 1200.0)
    th = Z2.Th / Z2.rho
    assert np.ptp(th) < 1e-9 * 300.0


def test_third_order_changes_only_the_explicit_terms():
    """With W carrying a cubic vertical profile, vorder = 3 changes the slow
    momentum tendencies (vertical advection and the centre value of W) but
    not the continuity and rho-theta tendencies, theta at the interfaces or
    Pi (the terms of the vertical system)."""
    m1, m3 = _model(1, hyper=False), _model(3, hyper=False)
    X = dc.initial_state(m1, 280.0, 1.0e5)
    rng = np.random.default_rng(5)
    zi = m1.vg.zi / m1.vg.zi[-1]
    X.W[:] = 0.02 * (zi * (1 - zi) * (0.5 + zi))[None, :] * (1 + 0.1 * rng.standard_normal((X.W.shape[0], 1)))
    X.M[:] = op.project_h(m1.rhat, rng.standard_normal(X.M.shape)) * X.rho[..., None]
    c1, c3 = dc.slow_terms(m1, X, 0.0), dc.slow_terms(m3, X, 0.0)
    for key in ("S_rho", "S_Th", "theta_i", "Pi", "p"):
        assert np.array_equal(c1[key], c3[key]), key
    assert np.abs(c1["S_M"] - c3["S_M"]).max() > 1e-12 * np.abs(c1["S_M"]).max()
    assert np.abs(c1["S_W"] - c3["S_W"]).max() > 0.0
