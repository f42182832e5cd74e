"""Pins of the oracle's shallow-atmosphere option (Sec. 3: 1/r replaced by
1/A with the traditional approximation; readings S-1..S-3): closed forms of
the geometry and of the Coriolis term, no vertical Coriolis and no
centripetal term, rest and mass invariants."""

import numpy as np

from conftest import oracle_grid
from oracle import diagnostics as dg
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls


def _model(shallow, omega=None, forcing="none", hyper=False, nv=6, glevel=3):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega if omega is None else omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    return dc.Model(oracle_grid(glevel, max_iter=10, tol=0.0), op.VerticalGrid(nv, 30.0e3, P.radius, shallow=shallow),
                    pl, forcing=forcing, hyperdiffusion=hyper, divergence_damping=hyper)


def test_shallow_geometry():
    m = _model(True)
    A = wls.EARTH.radius
    assert np.all(m.vg.rc == A) and np.all(m.vg.ri == A)
    V = dg.volumes(m)
    assert abs(V.sum() - 4 * np.pi * A ** 2 * 30.0e3) <= 1e-12 * V.sum()


def test_traditional_coriolis():
    """S_M(Omega) - S_M(0) = -proj(2 Omega sin(lat) r x M) for a small
    horizontal momentum on a resting column, and the vertical equation gets
    no Coriolis term at all."""
    om = 7.292e-5
    out = {}
    for o in (om, 0.0):
        m = _model(True, omega=o)
        X = dc.initial_state(m, 280.0, 1.0e5)
        noise = np.random.default_rng(3).standard_normal((m.grid.ncol, 1, 3))
        X.M[:] = 1e-4 * op.project_h(m.rhat, noise) * np.ones((1, m.vg.nv, 1))
        out[o] = dc.slow_terms(m, X, 0.0)
    r = m.rhat
    cor = 2 * om * r[:, 2][:, None, None] * np.cross(np.broadcast_to(r[:, None, :], X.M.shape), X.M)
    d = out[om]["S_M"] - out[0.0]["S_M"]
    np.testing.assert_allclose(d, -op.project_h(r, cor), rtol=0, atol=1e-12 * np.abs(cor).max())
    assert np.array_equal(out[om]["S_W"], out[0.0]["S_W"])


def test_no_centripetal_term():
    """A horizontal wind with W = 0 leaves the shallow vertical equation
    unchanged (w advected as a scalar is 0); the deep equation gets the
    centripetal force of the curved flow."""
    res = {}
    for shallow in (True, False):
        m = _model(shallow, omega=0.0)
        X0 = dc.initial_state(m, 280.0, 1.0e5)
        east = np.stack([-m.rhat[:, 1], m.rhat[:, 0], 0 * m.rhat[:, 0]], axis=-1)   # cos(lat) times east
        X1 = dc.State(X0.rho.copy(), X0.rho[..., None] * 20.0 * east[:, None, :], X0.W.copy(), X0.Th.copy())
        res[shallow] = dc.slow_terms(m, X1, 0.0)["S_W"] - dc.slow_terms(m, X0, 0.0)["S_W"]
    assert np.abs(res[True]).max() == 0.0
    assert np.abs(res[False][:, 1:-1]).max() > 1e-6


def test_rest_and_mass_in_the_shallow_atmosphere():
    m = _model(True, nv=10)
    X = dc.run(m, dc.initial_state(m, 300.0, 1.0e5), 5, 6, 1800.0)
    d = dg.diagnostics(m, X)
    assert d["max_vh"] < 1e-8 and d["max_w"] < 1e-8
    m = _model(True, forcing="held_suarez", hyper=True, nv=10)
    X = dc.initial_state(m, 300.0, 1.0e5, 0.1, np.random.default_rng(7).random((m.grid.ncol, 10)))
    m0 = dg.diagnostics(m, X)["mass"]
    X = dc.run(m, X, 5, 6, 1800.0)
    d = dg.diagnostics(m, X)
    assert abs(d["mass"] - m0) <= 1e-12 * m0 and d["max_vh"] > 1e-3
