"""Pins of the oracle's zonal band means (oracle/climate.py): closed forms of
solid-body rotation and of a zonal wave, and the band weights against the
layer volumes."""

import numpy as np

from conftest import oracle_grid
from oracle import climate as cl
from oracle import dycore as dc
from oracle import operators as op
from oracle.diagnostics import volumes
from oracle.grid import lonlat
import workloads as wls

NLAT = 18


def _model():
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
    return dc.Model(oracle_grid(4, max_iter=10, tol=0.0), op.VerticalGrid(6, 30.0e3, P.radius), pl)


def _with_wind(m, X, u_of, v_of):
    """X with the horizontal wind u east, v north (per column and level)."""
    lon, lat = lonlat(m.grid.points)
    east = np.stack([-np.sin(lon), np.cos(lon), np.zeros_like(lon)], axis=-1)
    north = np.stack([-np.sin(lat) * np.cos(lon), -np.sin(lat) * np.sin(lon), np.cos(lat)], axis=-1)
    vel = u_of(lon, lat)[..., None] * east[:, None, :] + v_of(lon, lat)[..., None] * north[:, None, :]
    return dc.State(X.rho.copy(), X.rho[..., None] * vel, X.W.copy(), X.Th.copy())


def test_band_weights_sum_to_the_layer_volume():
    m = _model()
    X = dc.initial_state(m, 280.0, 1.0e5)
    z = cl.zonal_band_means(m, X, NLAT)
    np.testing.assert_allclose(z[:, :, 0].sum(axis=1), volumes(m).sum(axis=0), rtol=1e-13)
    assert np.all(z[:, :, 0] > 0)
    # isothermal rest: u = v = 0, T = 280 K, no eddies
    assert np.abs(z[:, :, 1:3]).max() == 0 and np.abs(z[:, :, 5:]).max() < 1e-20
    np.testing.assert_allclose(z[:, :, 3], 280.0, rtol=1e-12)


def test_solid_body_rotation():
    """u = U cos(lat), v = 0: the band mean of u is the volume-weighted mean
    of U cos(lat) over the band (within the spread of the band's
    latitudes), v and the covariances with v vanish."""
    m = _model()
    X = _with_wind(m, dc.initial_state(m, 280.0, 1.0e5), lambda lo, la: 20.0 * np.cos(la)[:, None] * np.ones(6),
                   lambda lo, la: np.zeros((lo.size, 6)))
    z = cl.zonal_band_means(m, X, NLAT)
    edges = np.linspace(-np.pi / 2, np.pi / 2, NLAT + 1)
    lo_cos = np.minimum(np.cos(edges[:-1]), np.cos(edges[1:]))
    hi_cos = np.where((edges[:-1] < 0) & (edges[1:] > 0), 1.0, np.maximum(np.cos(edges[:-1]), np.cos(edges[1:])))
    assert np.all(z[:, :, 1] >= 20.0 * lo_cos - 1e-9) and np.all(z[:, :, 1] <= 20.0 * hi_cos + 1e-9)
    assert np.abs(z[:, :, 2]).max() < 1e-12 and np.abs(z[:, :, 5]).max() < 1e-12
    assert np.all(z[:, :, 7] >= -1e-12)


def test_zonal_wave_has_zero_mean_and_its_variance():
    """u = U cos(4 lon) at every latitude: zero zonal mean, eddy variance
    U^2/2 up to the grid's sampling of the wave (a few per cent on glevel 4),
    no v; v = U sin(lat) cos(2 lon) correlated with u gives [u'v'] near 0."""
    m = _model()
    U = 10.0
    X = _with_wind(m, dc.initial_state(m, 280.0, 1.0e5), lambda lo, la: U * np.cos(4 * lo)[:, None] * np.ones(6),
                   lambda lo, la: np.zeros((lo.size, 6)))
    z = cl.zonal_band_means(m, X, NLAT)
    mid = slice(2, NLAT - 2)                      # bands away from the poles hold many columns
    assert np.abs(z[:, mid, 1]).max() < 0.05 * U
    np.testing.assert_allclose(z[:, mid, 7], U * U / 2, rtol=0.1)
    assert np.abs(z[:, :, 8]).max() < 1e-20
