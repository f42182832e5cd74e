"""Pins of the oracle physics (Sec. 5-6) against closed-form special values of
the printed forcings. CPU only."""

import json
import os

import numpy as np
import pytest

from conftest import oracle_grid
from oracle import dycore as dc
from oracle import operators as op
from oracle import physics as ph
import workloads as wls

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "forcing_constants.json")))


def test_held_suarez_constants():
    g = GOLD["held_suarez"]
    assert ph.HS["k_f"] == pytest.approx(g["k_f_per_day"] / 86400.0)
    assert ph.HS["k_a"] == pytest.approx(g["k_a_per_day"] / 86400.0)
    assert ph.HS["k_s"] == pytest.approx(g["k_s_per_day"] / 86400.0)
    for k in ("sigma_b", "dT_y", "T_floor", "T_top"):
        assert ph.HS[k] == g[k]


def test_held_suarez_special_values():
    kappa = 287.0 / 1005.0
    p0 = 1.0e5
    # surface (sigma = 1, p = p0) at the equator and the pole
    Kv, KT, Teq = ph.held_suarez_coefficients(np.array([1.0, 1.0]), np.array([p0, p0]),
                                              np.array([0.0, np.pi / 2]), kappa)
    assert Teq[0] == pytest.approx(315.0, abs=1e-12)
    assert Teq[1] == pytest.approx(255.0, abs=1e-12)
    assert Kv[0] == pytest.approx(ph.HS["k_f"]) and Kv[1] == pytest.approx(ph.HS["k_f"])
    assert KT[0] == pytest.approx(ph.HS["k_s"])
    assert KT[1] == pytest.approx(ph.HS["k_a"])
    # above sigma_b there is no friction and K_T = k_a
    Kv, KT, Teq = ph.held_suarez_coefficients(np.array([0.7, 0.3]), np.array([7e4, 3e4]),
                                              np.array([0.3, -0.5]), kappa)
    assert np.all(Kv == 0.0) and np.allclose(KT, ph.HS["k_a"])
    # the stratosphere is clamped at 200 K
    Kv, KT, Teq = ph.held_suarez_coefficients(np.array([0.01]), np.array([1e3]), np.array([0.0]), kappa)
    assert Teq[0] == 200.0


def test_hot_jupiter_profile():
    h = GOLD["hot_jupiter"]
    assert ph.HJ["tau"] == h["tau_s"] and ph.HJ["z_stra"] == h["z_stra_m"]
    G, zs, dT, Ts = h["gamma_trop"], h["z_stra_m"], h["dT_stra"], h["T_surf"]
    # Eq. tvert at z = 0: Ts - G zs/2 + sqrt((G zs/2)^2 + dT^2); above z_stra: Ts - G zs + dT
    assert ph.hot_jupiter_T_vert(np.array(0.0)) == pytest.approx(Ts - G * zs / 2 + np.hypot(G * zs / 2, dT))
    assert ph.hot_jupiter_T_vert(np.array(3.0e6)) == pytest.approx(Ts - G * zs + dT)
    # continuous at z_stra
    assert ph.hot_jupiter_T_vert(np.array(zs * (1 - 1e-12))) == pytest.approx(
        ph.hot_jupiter_T_vert(np.array(zs * (1 + 1e-12))), abs=1e-6)
    # Eq. btrop: beta_trop(sigma = 1) = 1 below z_stra, 0 above; zero at sigma_stra
    assert ph.hot_jupiter_beta_trop(np.array(1.0), np.array(0.0)) == pytest.approx(1.0)
    assert ph.hot_jupiter_beta_trop(np.array(0.12), np.array(0.0)) == pytest.approx(0.0, abs=1e-15)
    assert ph.hot_jupiter_beta_trop(np.array(0.9), np.array(2.5e6)) == 0.0


def test_backward_euler_updates():
    """Eqs. im_eq_v / im_eq_t: momentum divided by (1 + K_v dt); T relaxes
    toward T_eq; rho unchanged; surface pressure recovers p_surf for the
    discretely balanced isothermal column."""
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    G = oracle_grid(2, max_iter=10, tol=0.0)
    m = dc.Model(G, op.VerticalGrid(12, 30.0e3, P.radius), pl, forcing="held_suarez")
    X = dc.initial_state(m, 300.0, 1.0e5)
    p = dc.pressure(pl, X.Th)
    T = dc.temperature(pl, X.rho, p)
    assert np.allclose(ph.surface_pressure(m, p, T), 1.0e5, rtol=1e-13)
    X.M[:] = op.project_h(m.rhat, np.ones_like(X.M))
    dt = 1800.0
    Y = ph.apply_physics(m, X, dt)
    sigma = p / 1.0e5
    from oracle.grid import lonlat
    lon, lat = lonlat(G.points)
    Kv, KT, Teq = ph.held_suarez_coefficients(sigma, p, lat[:, None], pl.kappa)
    assert np.allclose(Y.M, X.M / (1 + Kv * dt)[..., None], rtol=1e-14)
    Tn = dc.temperature(pl, Y.rho, dc.pressure(pl, Y.Th))
    assert np.allclose(Tn, (T + KT * dt * Teq) / (1 + KT * dt), rtol=1e-12)
    assert np.array_equal(Y.rho, X.rho) and np.array_equal(Y.W, X.W)
