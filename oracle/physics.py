"""Oracle physics core (Sec. 5, PROFX) with the Sec. 6 forcings, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

After each large step the physics applies the backward-Euler updates
Eq. im_eq_v (boundary-layer friction on rho v_h) and Eq. im_eq_t (Newtonian
relaxation of T), with the same dt as the large step. rho is not touched;
rho theta is recomputed from the new T at fixed rho (ideal gas + Eq.
pressure). W is not touched.

Readings:

* sigma = p / p_s with p_s extrapolated from the lowest layer centre to z = 0
  with the hydrostatic equation at that layer's constant temperature:
  p_s = p_0 exp(g z_0 / (Rd T_0)) (Sec. 5).
* Held-Suarez T_eq and K_T (Sec. 6.1): the paper does not define
  (Delta theta)_z and p*, and its K_T lacks the "max"; we take them from the
  Held and Suarez (1994) definition that Sec. 6.1 cites: (Delta theta)_z = 10 K,
  p* = 1e5 Pa (= p0), K_T = k_a + (k_s - k_a) max(0, (sigma - sigma_b)/(1 - sigma_b)) cos^4 phi.
  The log is natural. One Earth day is 86400 s.
* Hot Jupiter (Sec. 6.2, Eqs. teq-hj, btrop, tvert) as printed: beta_trop is
  the sine of sigma below z_stra (even where sigma < sigma_stra) and 0
  above; K_v = 0; K_T = 1/tau with tau = 1.5e5 s. The sub-stellar point is at
  longitude 0 (the paper's is shifted by pi, which only moves the pattern).
  The factor cos(lambda) cos(phi) of Eq. teq-hj is evaluated as the x
  coordinate of the unit position vector, which it equals exactly; at the
  poles the longitude is undefined and the factor is 0.
"""

import numpy as np

from . import dycore as dc
from .grid import lonlat

DAY = 86400.0

HS = dict(k_f=1.0 / DAY, k_a=1.0 / (40.0 * DAY), k_s=1.0 / (4.0 * DAY), sigma_b=0.7,
          dT_y=60.0, dtheta_z=10.0, p0=1.0e5, T_floor=200.0, T_top=315.0)

HJ = dict(sigma_stra=0.12, z_stra=2.0e6, T_surf=1600.0, gamma_trop=2.0e-4, dT_stra=10.0,
          tau=1.5e5)


def surface_pressure(model, p, T):
    """Sec. 5: hydrostatic extrapolation at constant T from the lowest layer."""
    g, Rd = model.planet.gravity, model.planet.Rd
    return p[:, 0] * np.exp(g * model.vg.zc[0] / (Rd * T[:, 0]))


def held_suarez_coefficients(sigma, p, lat, kappa):
    """Eq. im_eq_fv and the Sec. 6.1 T_eq, K_T. Returns (K_v, K_T, T_eq)."""
    h = HS
    ramp = np.maximum(0.0, (sigma - h["sigma_b"]) / (1.0 - h["sigma_b"]))
    K_v = h["k_f"] * ramp
    K_T = h["k_a"] + (h["k_s"] - h["k_a"]) * ramp * np.cos(lat) ** 4
    T_eq = np.maximum(h["T_floor"],
                      (h["T_top"] - h["dT_y"] * np.sin(lat) ** 2
                       - h["dtheta_z"] * np.log(p / h["p0"]) * np.cos(lat) ** 2)
                      * (p / h["p0"]) ** kappa)
    return K_v, K_T, T_eq


def hot_jupiter_T_vert(z):
    """Eq. tvert."""
    h = HJ
    zs, G, dT = h["z_stra"], h["gamma_trop"], h["dT_stra"]
    below = h["T_surf"] - G * (zs + (z - zs) / 2.0) + np.sqrt((G * (z - zs) / 2.0) ** 2 + dT ** 2)
    above = h["T_surf"] - G * zs + dT
    return np.where(z <= zs, below, above)


def hot_jupiter_beta_trop(sigma, z):
    """Eq. btrop."""
    h = HJ
    s = np.sin(np.pi * (sigma - h["sigma_stra"]) / (2.0 * (1.0 - h["sigma_stra"])))
    return np.where(z <= h["z_stra"], s, 0.0)


def hot_jupiter_coefficients(sigma, z, coslon_coslat, dT_ep):
    """Eq. teq-hj with K_v = 0, K_T = 1/tau. Returns (K_v, K_T, T_eq)."""
    T_eq = hot_jupiter_T_vert(z) + hot_jupiter_beta_trop(sigma, z) * dT_ep * coslon_coslat
    return np.zeros_like(sigma), np.full_like(sigma, 1.0 / HJ["tau"]), T_eq


def apply_physics(model, X, dt):
    """Eqs. im_eq_v and im_eq_t (backward Euler, Sec. 5)."""
    if model.forcing == "none":
        return X
    pl = model.planet
    p = dc.pressure(pl, X.Th)
    T = dc.temperature(pl, X.rho, p)
    ps = surface_pressure(model, p, T)
    sigma = p / ps[:, None]
    lon, lat = lonlat(model.grid.points)
    if model.forcing == "held_suarez":
        K_v, K_T, T_eq = held_suarez_coefficients(sigma, p, lat[:, None], pl.kappa)
    elif model.forcing == "hot_jupiter":
        K_v, K_T, T_eq = hot_jupiter_coefficients(sigma, model.vg.zc[None, :],
                                                  model.grid.points[:, 0:1], model.hj_dT)
    else:
        raise ValueError(model.forcing)
    M = X.M / (1.0 + K_v * dt)[..., None]
    T_new = (T + K_T * dt * T_eq) / (1.0 + K_T * dt)
    Th = dc.rhotheta_from_p(pl, X.rho * pl.Rd * T_new)
    return dc.State(X.rho.copy(), M, X.W.copy(), Th)
