"""A textbook wave against the oracle's whole large step: the Lamb wave.

Linearised about an isothermal atmosphere at rest without rotation, a
horizontally propagating acoustic mode with no vertical motion exists (the
Lamb wave): w = 0 requires the perturbation to be hydrostatic, dp'/dz = -g rho',
and adiabatic, p' = c^2 rho' with c^2 = gamma R_d T, so
p' ~ exp(-g z / c^2) Y_l(lat, lon); on a sphere of radius a it oscillates at
omega = c sqrt(l (l + 1)) / a. For l = 1 and T = 300 K the period is about
22.6 hours. The split-explicit scheme carries this mode in its horizontally
explicit acoustic small steps (Eqs. mom2 and pt2); the measured period must
approach the analytic one at second order in the grid spacing, and the
amplitude must survive half a period (the divergence damping, which acts on
exactly this divergent motion, and the hyperdiffusion are off). A wrong
factor in the pressure gradient or the divergence (a missing 1/r, a gamma
for a kappa) shifts the period by far more than the 1% allowed."""

import numpy as np

from conftest import oracle_grid
from oracle import dycore as dc
from oracle import operators as op
from oracle.diagnostics import volumes
import workloads as wls


def _lamb_wave(glevel, nv=10, z_top=10.0e3, dt=1800.0, n_large=36, eps=1e-4, T0=300.0):
    P = wls.EARTH
    pl = dc.Planet(P.radius, 0.0, P.gravity, P.Rd, P.cp, P.p_ref, 0.0)
    vg = op.VerticalGrid(nv, z_top, P.radius)
    m = dc.Model(oracle_grid(glevel, max_iter=200, tol=1e-6), vg, pl, hyperdiffusion=False,
                 divergence_damping=False)
    X0 = dc.initial_state(m, T0, 1.0e5)
    p_bg = dc.pressure(pl, X0.Th)
    c2 = pl.gamma * pl.Rd * T0
    Y1 = m.rhat[:, 2][:, None]                                          # sin(lat), l = 1
    p1 = eps * 1.0e5 * np.exp(-pl.gravity * vg.zc / c2)[None, :] * Y1
    X = dc.State(X0.rho + p1 / c2, X0.M.copy(), X0.W.copy(), dc.rhotheta_from_p(pl, p_bg + p1))
    V = volumes(m)
    amplitude = lambda S: np.sum(V * (dc.pressure(pl, S.Th) - p_bg) * Y1) / np.sum(V * p1 * Y1)
    a = [amplitude(X)]
    for _ in range(n_large):
        X = dc.large_step(m, X, dt, 6)
        a.append(amplitude(X))
    a, t = np.array(a), dt * np.arange(n_large + 1)
    zeros = [t[i] - a[i] * dt / (a[i + 1] - a[i]) for i in range(n_large) if a[i] * a[i + 1] < 0]
    period = 2.0 * (zeros[1] - zeros[0])                                # from T/4 to 3T/4
    analytic = 2.0 * np.pi * P.radius / (np.sqrt(c2) * np.sqrt(2.0))
    return period / analytic, a.min()


def test_lamb_wave_period_converges_at_second_order():
    r3, min3 = _lamb_wave(3)
    r4, min4 = _lamb_wave(4)
    assert abs(r3 - 1.0) < 0.015 and abs(r4 - 1.0) < 0.005, (r3, r4)
    assert abs(r3 - 1.0) / abs(r4 - 1.0) > 2.5, (r3, r4)
    assert min3 < -0.98 and min4 < -0.98, (min3, min4)                 # half a period later, reversed
