"""Oracle energy fixer and budgets, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3 (after Eq. pressure): the entropy equation does not return the kinetic
energy lost at the truncation scale to the thermal energy, and the model has
a scheme after Williamson (2009) that restores the balance by adjusting the
internal energy by the same amount at every grid point; the simulations of
Sec. 6 were run without it. The paper gives no formula. Reading F-1: once per
large step, after the three RK3 stages of the dynamics and before the physics
(whose heating and friction are the physical sources), the temperature of
every cell is raised by one value dT chosen so that the total energy of
``diagnostics.diagnostics`` (internal + kinetic + potential, Sec. 3) equals its
value at the start of the step; the density and momentum are unchanged and
rho theta follows from Eq. pressure at the new temperature. Since the
internal energy is rho c_v T per unit volume, dT = (E_start - E_dyn) /
(c_v * sum V rho).
"""

import numpy as np

from . import dycore as dc
from .diagnostics import diagnostics, volumes


def energy_fix(model, X_start, X_dyn):
    """X_dyn with the uniform temperature adjustment of reading F-1 that
    restores the total energy of X_start; returns (state, dT)."""
    pl = model.planet
    e_start = diagnostics(model, X_start)["energy"]
    e_dyn = diagnostics(model, X_dyn)["energy"]
    mass = float(np.sum(volumes(model) * X_dyn.rho))
    dT = (e_start - e_dyn) / (pl.cv * mass)
    T = dc.temperature(pl, X_dyn.rho, dc.pressure(pl, X_dyn.Th))
    Th = dc.rhotheta_from_p(pl, X_dyn.rho * pl.Rd * (T + dT))
    return dc.State(X_dyn.rho.copy(), X_dyn.M.copy(), X_dyn.W.copy(), Th), dT


def budget_row(model, X_start, X_dyn, dT):
    """One large step's budget: mass, total energy and axial angular momentum
    at the start of the step and after its dynamics (before any fix), and the
    fixer's dT (0 without it)."""
    a, b = diagnostics(model, X_start), diagnostics(model, X_dyn)
    return [a["mass"], a["energy"], a["aam"], b["mass"], b["energy"], b["aam"], dT, 0.0]
