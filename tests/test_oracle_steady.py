"""A steady solution of the continuous equations against the oracle's whole
large step: rigid rotation of an isothermal atmosphere.

In the frame that rotates with Omega, air turning with an extra angular
velocity w about the same axis (u = w s eastward, s the distance from the
axis, W = 0) feels the Coriolis and centripetal accelerations together as
(2 Omega w + w^2) s outward from the axis. With gravity constant and radial
(Sec. 3) both body forces are gradients, g r and (2 Omega w + w^2) s^2 / 2, so
an isothermal ideal gas with

    ln p = (-g z + (2 Omega w + w^2) s^2 / 2) / (R_d T) + const

is in exact balance and stays at rest in the rotating frame for all time.
The discrete model holds it up to its truncation error: the horizontal
momentum must change by less and less as the grid is refined, at second
order (Sec. 2: the modified grid's operators). A dropped or mis-signed
Coriolis, centripetal or pressure-gradient term leaves an imbalance that
does not shrink with the grid (with the Coriolis term dropped the momentum
changes by 7% in two steps at every grid level)."""

import numpy as np

from conftest import oracle_grid
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls


def _rigid_rotation_change(glevel, w=1e-5, nv=8, steps=2):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    vg = op.VerticalGrid(nv, 12.0e3, P.radius)
    m = dc.Model(oracle_grid(glevel, max_iter=200, tol=1e-6), vg, pl, hyperdiffusion=False,
                 divergence_damping=False)
    T = 280.0
    r = m.rhat
    s2 = (r[:, 0] ** 2 + r[:, 1] ** 2)[:, None] * vg.rc[None, :] ** 2
    k = 2.0 * pl.omega * w + w * w
    p = 1e5 * np.exp((-pl.gravity * vg.zc[None, :] + 0.5 * k * (s2 - P.radius ** 2)) / (pl.Rd * T))
    rho = p / (pl.Rd * T)
    east_s = np.stack([-r[:, 1], r[:, 0], 0.0 * r[:, 0]], axis=-1)       # s / r times the unit east vector
    vel = w * vg.rc[None, :, None] * east_s[:, None, :]                 # w s east
    X = dc.State(rho, rho[..., None] * vel, np.zeros((m.grid.ncol, nv + 1)), dc.rhotheta_from_p(pl, p))
    Y = dc.run(m, X, steps, 6, 600.0)
    return np.linalg.norm(Y.M - X.M) / np.linalg.norm(X.M)


def test_rigid_rotation_is_held_at_second_order():
    e3, e4, e5 = (_rigid_rotation_change(g) for g in (3, 4, 5))
    assert e3 < 3e-3, (e3, e4, e5)
    assert e3 / e4 > 3.0 and e4 / e5 > 3.0, (e3, e4, e5)
