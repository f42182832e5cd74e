"""Pins of the oracle's hydrostatic switch (Sec. 3: the vertical pressure
gradient balances gravity; reading H1). The balance itself is checked with
the hydrostatic equation written out here on the model's own levels, with
the pressure from the equation of state, so that a term left in the
vertical system (the identity, W*, the vertical advection or Coriolis, the
diffusion of W) shows up as a residual of first order in the departure from
balance instead of second order."""

import numpy as np

from conftest import oracle_grid
from oracle import diagnostics as dg
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls


def _model(hydrostatic, forcing="none", hyper=False, nv=10, glevel=2, omega=None):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega if omega is None else omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    return dc.Model(oracle_grid(glevel, max_iter=10, tol=0.0), op.VerticalGrid(nv, 30.0e3, P.radius), pl,
                    forcing=forcing, hyperdiffusion=hyper, divergence_damping=hyper, hydrostatic=hydrostatic)


def _imbalance(m, X):
    """dp/dz + g rho at the interior interfaces, relative to g rho there:
    centred difference of the equation-of-state pressure over the centres'
    spacing, rho linearly interpolated in z to the interface."""
    zc, zi = m.vg.zc, m.vg.zi
    p = m.planet.p_ref * (m.planet.Rd * X.Th / m.planet.p_ref) ** (m.planet.cp / (m.planet.cp - m.planet.Rd))
    t = (zi[1:-1] - zc[:-1]) / (zc[1:] - zc[:-1])
    rho_i = (1 - t) * X.rho[:, :-1] + t * X.rho[:, 1:]
    dpdz = (p[:, 1:] - p[:, :-1]) / (zc[1:] - zc[:-1])
    return np.abs(dpdz + m.planet.gravity * rho_i).max() / (m.planet.gravity * rho_i).max()


def _perturbed(m, eps, wind=0.0):
    """Resting balanced state with rho theta scaled by (1 + eps sin) in the
    vertical (horizontally uniform), plus an optional solid-body zonal wind."""
    X = dc.initial_state(m, 280.0, 1.0e5)
    s = np.sin(np.pi * m.vg.zc / m.vg.zi[-1])
    X.Th *= 1.0 + eps * s[None, :]
    if wind:
        east = np.stack([-m.rhat[:, 1], m.rhat[:, 0], 0 * m.rhat[:, 0]], axis=-1)   # cos(lat) times east
        X.M[:] = X.rho[..., None] * wind * east[:, None, :]
    return X


def test_initial_state_is_balanced():
    m = _model(True)
    assert _imbalance(m, dc.initial_state(m, 280.0, 1.0e5)) < 1e-12


def _one_small_step(m, X, dtau):
    co = dc.slow_terms(m, X, 0.0)
    pert = dict(rho=0 * X.rho, M=0 * X.M, W=0 * X.W, Th=X.Th.copy(), p=dc.pressure(m.planet, X.Th) - co["p"])
    q = dc.small_step(m, X, co, pert, dtau, 0.0)
    return dc.State(X.rho + q["rho"], X.M + q["M"], X.W + q["W"], q["Th"])


def test_one_small_step_restores_balance_to_second_order():
    """From a column out of balance by eps, one hydrostatic small step leaves
    an imbalance of order eps^2 (the linearised p* of reading R3): halving
    eps quarters it, and it does not depend on dtau (W is diagnosed, so
    dtau W, the displacement, is what the balance fixes). The
    nonhydrostatic step keeps an imbalance of order eps that grows as dtau
    shrinks (the column only starts to accelerate)."""
    res = {}
    for eps in (2e-3, 1e-3):
        for hyd in (True, False):
            m = _model(hyd)
            X0 = _perturbed(m, eps)
            res[eps, hyd] = [_imbalance(m, X0)] + [_imbalance(m, _one_small_step(m, X0, d)) for d in (200.0, 20.0)]
    r0, h200, h20 = res[2e-3, True]
    assert r0 > 1e-3 and h200 < 1e-3 * r0, res
    assert abs(h20 - h200) <= 1e-3 * h200, res
    assert 3.9 < h200 / res[1e-3, True][1] < 4.1, res
    n200, n20 = res[2e-3, False][1:]
    assert n20 > 0.1 * r0 and n200 > 10 * h200, res
    assert 1.9 < n20 / res[1e-3, False][2] < 2.1, res


def test_hydrostatic_large_step_converges_to_balance():
    """Every small step is one Newton step on the nonlinear balance, so after
    the ten small steps of a large step the column is balanced to rounding;
    the implicit nonhydrostatic model damps its acoustic oscillation but is
    still out of balance by orders of magnitude more."""
    for hyd, bound in ((True, 1e-12), (False, None)):
        m = _model(hyd)
        r = _imbalance(m, dc.large_step(m, _perturbed(m, 2e-3), 600.0, 6))
        if hyd:
            assert r < bound, r
            rh = r
        else:
            assert r > 1e3 * rh, (r, rh)


def test_hydrostatic_balance_with_motion():
    """A 40 m/s solid-body wind with rotation: the nonhydrostatic vertical
    equation balances the radial advection (centripetal) and Coriolis parts,
    of relative size (u^2/r + 2 Omega u cos(lat)) / g ~ 6e-4, against dp/dz +
    g rho; the hydrostatic one has neither, so its column stays in balance."""
    r = {}
    for hyd in (True, False):
        m = _model(hyd)
        r[hyd] = _imbalance(m, dc.large_step(m, _perturbed(m, 1e-3, wind=40.0), 600.0, 6))
    assert r[True] < 1e-7 and 3e-4 < r[False] < 1.2e-3, r


def test_rest_stays_at_rest_and_mass():
    m = _model(True, forcing="held_suarez", hyper=True)
    X0 = dc.initial_state(m, 280.0, 1.0e5)
    X = dc.run(m, X0, 3, 6, 600.0)
    assert np.abs(X.M / X.rho[..., None]).max() < 5.0       # only the forcing moves air
    v = dg.volumes(m)
    assert abs((v * X.rho).sum() - (v * X0.rho).sum()) <= 1e-12 * (v * X0.rho).sum()
    Xr = dc.run(_model(True), dc.initial_state(_model(True), 280.0, 1.0e5), 3, 6, 600.0)
    assert np.abs(Xr.M).max() < 1e-8 and np.abs(Xr.W).max() < 1e-8


def test_switch_off_is_the_nonhydrostatic_model():
    """delta = 1 reproduces the default model exactly; delta = 0 changes W
    far more than the horizontal momentum of a large-scale flow (H / L << 1,
    the approximation's premise)."""
    mh, mn = _model(True), _model(False)
    X0 = _perturbed(mn, 1e-4, wind=20.0)
    rng = np.random.default_rng(4)
    X0.Th *= 1.0 + 1e-4 * rng.standard_normal(X0.Th.shape[0])[:, None]
    a = dc.large_step(mn, X0, 600.0, 6)
    b = dc.large_step(dc.Model(mn.grid, mn.vg, mn.planet, hyperdiffusion=False, divergence_damping=False),
                      X0, 600.0, 6)
    assert np.array_equal(a.W, b.W) and np.array_equal(a.M, b.M)
    h = dc.large_step(mh, X0, 600.0, 6)
    dM = np.abs(h.M - a.M).max() / np.abs(a.M).max()
    dW = np.abs(h.W - a.W).max() / np.abs(a.W).max()
    assert 0 < dM < 1e-2 and dW > 10 * dM, (dM, dW)


def test_held_suarez_start_profile():
    """Sec. 6.1's start: every layer at the equatorial T_eq of its own
    pressure (written out here: max(200 K, (315 K - 10 K ln(p / 1e5 Pa))
    (p / 1e5 Pa)^kappa)), the column in discrete hydrostatic balance, the
    same profile in every column, at rest; near the ground T_eq is about
    315 K and the top of a 30 km column is on the 200 K floor."""
    m = _model(False, nv=30)
    X = dc.initial_state(m, 0.0, 1.0e5, profile="held_suarez")
    pl = m.planet
    p = dc.pressure(pl, X.Th)
    T = p / (pl.Rd * X.rho)
    kappa = pl.Rd / pl.cp
    T_eq = np.maximum(200.0, (315.0 - 10.0 * np.log(p / 1e5)) * (p / 1e5) ** kappa)
    assert np.abs(T - T_eq).max() < 1e-9
    assert _imbalance(m, X) < 1e-12
    assert np.abs(T - T[:1]).max() == 0.0 and not X.M.any() and not X.W.any()
    assert 300.0 < T[0, 0] < 316.0 and abs(T[0, -1] - 200.0) < 1e-9
    # and it stays at rest without forcing
    Y = dc.run(_model(False, nv=30), X, 2, 6, 600.0)
    assert np.abs(Y.M).max() < 1e-8 * np.abs(Y.rho).max() and np.abs(Y.W).max() < 1e-8
