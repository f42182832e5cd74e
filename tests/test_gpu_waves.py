"""The CUDA path against solutions of the continuous equations, without the
oracle in between: the Lamb wave of an isothermal atmosphere (an l = 1
acoustic mode with no vertical motion, p' ~ exp(-g z / c^2) sin(lat),
period 2 pi a / (c sqrt 2)) and rigid rotation of an isothermal atmosphere in
gradient balance (steady). The states are built here from the library's own
resting start, its grid points and its level heights (uniform layers)."""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
import workloads as wls

NV, Z_TOP, T0 = 10, 10.0e3, 300.0


def _setup(glevel, precision, omega):
    P = wls.EARTH
    grid = thor.thor_grid_create(glevel, NV, P.radius, Z_TOP, thor.thor_spring(1.15, 1.0, 1.0, 0.01, 1e-6, 200))
    planet = thor.thor_planet(P.radius, omega, P.gravity, P.Rd, P.cp, P.p_ref, 0.0)
    init = thor.thor_init(T0, 1.0e5, 0.0, 1, thor.THOR_FORCING_NONE, 0.0, precision, 0, 0, 0, 0, 0)
    st = thor.thor_state_init(grid, planet, init)
    ncol = thor.thor_grid_info(grid)["ncol"]
    zc = (np.arange(NV) + 0.5) * Z_TOP / NV
    return P, grid, st, ncol, zc


def _rhotheta(P, p):
    return P.p_ref / P.Rd * (p / P.p_ref) ** ((P.cp - P.Rd) / P.cp)


@pytest.mark.parametrize("precision", [thor.THOR_FP64, thor.THOR_MIXED])
def test_lamb_wave_period(precision):
    periods = []
    for glevel in (4, 5):
        P, grid, st, ncol, zc = _setup(glevel, precision, 0.0)
        try:
            rho, mom, w, th = thor.thor_state_get_all(st, ncol, NV)
            p_bg = thor.thor_state_get(st, thor.THOR_FIELD_PRESSURE, ncol, NV)
            c2 = P.cp / (P.cp - P.Rd) * P.Rd * T0
            y1 = thor.thor_grid_points(grid)[:, 2][:, None]
            p1 = 1e-4 * 1.0e5 * np.exp(-P.gravity * zc / c2)[None, :] * y1
            thor.thor_state_set_all(st, rho + p1 / c2, mom, w, _rhotheta(P, p_bg + p1))
            weight = thor.thor_grid_areas(grid)[:, None] * ((P.radius + zc) ** 2)[None, :] * y1
            norm = np.sum(weight * p1)
            dt, n = 1800.0, 36
            a = [1.0]
            for _ in range(n):
                thor.thor_step(st, 1, 6, dt)
                a.append(np.sum(weight * (thor.thor_state_get(st, thor.THOR_FIELD_PRESSURE, ncol, NV) - p_bg)) / norm)
            a = np.array(a)
            z = [dt * (i - a[i] / (a[i + 1] - a[i])) for i in range(n) if a[i] * a[i + 1] < 0]
            periods.append(2.0 * (z[1] - z[0]) / (2.0 * math.pi * P.radius / math.sqrt(2.0 * c2)))
            assert a.min() < -0.98, a.min()
        finally:
            thor.thor_state_destroy(st)
            thor.thor_grid_destroy(grid)
    r4, r5 = periods
    assert abs(r4 - 1.0) < 0.005 and abs(r5 - 1.0) < 0.002, periods
    assert abs(r4 - 1.0) > 2.0 * abs(r5 - 1.0), periods


def test_rigid_rotation_is_steady():
    """u = w s eastward with ln p = (-g z + (2 Omega w + w^2) s^2 / 2) / (R_d T):
    the momentum changes by less than 1e-3 (relative) in two large steps at
    glevel 4 and by a quarter of that at glevel 5."""
    change = []
    wrot, omega = 1e-5, wls.EARTH.omega
    for glevel in (4, 5):
        P, grid, st, ncol, zc = _setup(glevel, thor.THOR_FP64, omega)
        try:
            r = thor.thor_grid_points(grid)
            rc = P.radius + zc
            s2 = (r[:, 0] ** 2 + r[:, 1] ** 2)[:, None] * rc[None, :] ** 2
            k = 2.0 * omega * wrot + wrot * wrot
            p = 1.0e5 * np.exp((-P.gravity * zc[None, :] + 0.5 * k * (s2 - P.radius ** 2)) / (P.Rd * T0))
            rho = p / (P.Rd * T0)
            east_s = np.stack([-r[:, 1], r[:, 0], 0.0 * r[:, 0]], axis=-1)
            mom = rho[..., None] * wrot * rc[None, :, None] * east_s[:, None, :]
            thor.thor_state_set_all(st, rho, np.ascontiguousarray(mom), np.zeros((ncol, NV + 1)), _rhotheta(P, p))
            m0 = thor.thor_state_get(st, thor.THOR_FIELD_MOM, ncol, NV)
            thor.thor_step(st, 2, 6, 600.0)
            m1 = thor.thor_state_get(st, thor.THOR_FIELD_MOM, ncol, NV)
            change.append(np.linalg.norm(m1 - m0) / np.linalg.norm(m0))
        finally:
            thor.thor_state_destroy(st)
            thor.thor_grid_destroy(grid)
    assert change[0] < 1e-3 and change[0] > 3.0 * change[1], change
