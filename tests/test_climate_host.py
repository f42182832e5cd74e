"""Host-side post-processing of the climate runner (paper_1607_05535_gb300.
climate.summarize) on synthetic band means with known answers: the jets'
position, the mass stream function of a uniform northward wind (Sec. 6.1:
Psi = 2 pi A cos(lat) / g times the integral of [v] over pressure from the
top), the sign conventions of the eddy fluxes, and the pressure-level
fields. No GPU."""

import math

import numpy as np

from paper_1607_05535_gb300 import climate


def _means(nv=10, nlat=18, dp=9.0e3, p0=9.5e4):
    m = np.zeros((nv, nlat, 9))
    p = p0 - dp * np.arange(nv)
    m[..., 0] = 1.0
    m[..., 3] = 250.0
    m[..., 4] = p[:, None]
    return m, p


def test_jets_and_surface_winds():
    m, p = _means()
    lat = (np.arange(18) + 0.5) * 10.0 - 90.0
    m[6, 13, 1] = 31.0                       # north jet at band 13 (45 deg), level 6
    m[7, 4, 1] = 27.0                        # south jet at band 4 (-45 deg), level 7
    m[0, :, 1] = np.where(np.abs(lat) < 30, -3.0, 2.0)
    s = climate.summarize(m, 6.371e6, 9.8)
    assert s["jets"]["north"] == {"u_ms": 31.0, "lat_deg": lat[13], "p_hPa": p[6] / 100.0, "level": 6}
    assert s["jets"]["south"]["u_ms"] == 27.0 and s["jets"]["south"]["lat_deg"] == lat[4]
    assert s["surface_u_equator_ms"] == -3.0 and s["surface_u_poleward_60_ms"] == 2.0


def test_stream_function_of_a_uniform_northward_wind():
    """A northward wind v0 in one band at every level: Psi grows from the top
    down to 2 pi A cos(lat) v0 (total pressure thickness) / g at the lowest
    level; the level thicknesses of uniform spacing dp add up to nv dp."""
    nv, dp, A, g, v0 = 10, 9.0e3, 6.371e6, 9.8, 1.5
    m, p = _means(nv=nv, dp=dp)
    b = 12
    lat = (b + 0.5) * 10.0 - 90.0
    m[:, b, 2] = v0
    s = climate.summarize(m, A, g)
    expect = 2.0 * math.pi * A * math.cos(math.radians(lat)) * v0 * nv * dp / g
    assert abs(s["psi_max_kg_s"] - expect) <= 1e-12 * expect
    assert s["psi_max_lat_deg"] == lat and s["psi_min_kg_s"] == 0.0


def test_eddy_flux_conventions_and_pressure_levels():
    m, p = _means()
    lat = (np.arange(18) + 0.5) * 10.0 - 90.0
    m[:, lat > 0, 5] = np.linspace(0.0, 20.0, 10)[:, None]    # poleward momentum flux, north
    m[:, lat < 0, 5] = -np.linspace(0.0, 20.0, 10)[:, None]   # poleward momentum flux, south
    m[:, :, 1] = (1.0e5 - p[:, None]) * 1e-3                   # u linear in p
    s = climate.summarize(m, 6.371e6, 9.8, p_levels=np.array([9.0e4, 5.0e4, 1.0e3]))
    assert s["eddy_uv_north_max"] == 20.0 and s["eddy_uv_south_min"] == -20.0
    u = np.array(s["u_p_levels"], dtype=object)
    assert abs(u[0][0] - 10.0) < 1e-9 and abs(u[1][5] - 50.0) < 1e-9 and u[2][0] is None   # 10 hPa above the top
