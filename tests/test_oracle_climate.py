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
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
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


def test_w_star_vanishes_for_band_constant_fields_and_is_linear():
    """[w*] is zero where [w] is constant over every band and level, it has a
    zero volume-weighted mean in every band, and w* of a sum is the sum."""
    m = _model()
    band = cl.band_of(m.grid.points, NLAT)
    rng = np.random.default_rng(2)
    per_band = rng.standard_normal((NLAT, m.vg.nv))
    ws = cl.w_star(m, per_band[band], NLAT)
    assert np.abs(ws).max() <= 1e-14 * np.abs(per_band).max()      # rounding of the weighted sums
    a, b = rng.standard_normal((2, m.grid.ncol, m.vg.nv))
    wa, wb = cl.w_star(m, a, NLAT), cl.w_star(m, b, NLAT)
    np.testing.assert_allclose(cl.w_star(m, a + b, NLAT), wa + wb, atol=1e-14)
    V = volumes(m)
    for k in range(m.vg.nv):
        s = np.bincount(band, weights=V[:, k] * wa[:, k], minlength=NLAT)
        assert np.abs(s).max() <= 1e-13 * np.abs(V[:, k] * wa[:, k]).sum()
    # a band-constant part added to a field leaves its map unchanged
    np.testing.assert_allclose(cl.w_star(m, a + per_band[band], NLAT), wa, atol=1e-14)


def test_cell_w_of_a_linear_profile():
    """W linear in height with a uniform density: the centre value is exact
    (Lagrange k = 1 reproduces a linear function), w = (a + b z_c) / rho."""
    m = _model()
    X = dc.initial_state(m, 280.0, 1.0e5)
    X.rho[:] = 1.2
    X.W[:] = 0.3 + 2e-5 * m.vg.zi[None, :]
    np.testing.assert_allclose(cl.cell_w(m, X), (0.3 + 2e-5 * m.vg.zc[None, :]) / 1.2 * np.ones_like(X.rho),
                               rtol=1e-14)


def test_pressure_levels_linear_and_bounds():
    """A field linear in p comes back exactly at any target inside a band's
    pressure range (whichever way the levels are ordered), the model levels'
    own pressures return the level values, and targets outside are NaN."""
    rng = np.random.default_rng(5)
    nv, nlat = 8, 5
    p = np.sort(rng.uniform(1e3, 1e5, (nv, nlat)), axis=0)[::-1]      # decreasing with height
    f = 3.0 - 2e-4 * p
    targets = np.array([2e5, 9e4, 5e4, 2e4, 5e3, 10.0])
    out = cl.to_pressure_levels(f, p, targets)
    for b in range(nlat):
        for i, pt in enumerate(targets):
            if p[:, b].min() <= pt <= p[:, b].max():
                assert abs(out[i, b] - (3.0 - 2e-4 * pt)) <= 1e-12
            else:
                assert np.isnan(out[i, b])
    g = rng.standard_normal((nv, nlat))
    for b in range(nlat):
        np.testing.assert_allclose(cl.to_pressure_levels(g[:, b:b + 1], p[:, b:b + 1], p[:, b])[:, 0], g[:, b],
                                   rtol=1e-13)


def test_runner_post_processing_matches_the_oracle():
    """The climate runner's [w*] and pressure-level interpolation (numpy on
    the host, written apart from the oracle) against the oracle's on the same
    inputs; the runner weights a level by area, the oracle by volume."""
    climate = __import__("paper_1607_05535_gb300.climate", fromlist=["w_star"])
    m = _model()
    rng = np.random.default_rng(8)
    wm = rng.standard_normal((m.grid.ncol, m.vg.nv))
    np.testing.assert_allclose(climate.w_star(wm, m.grid.points, m.grid.area, NLAT), cl.w_star(m, wm, NLAT),
                               atol=1e-13)
    np.testing.assert_array_equal(climate.bands(m.grid.points, NLAT), cl.band_of(m.grid.points, NLAT))
    nv, nlat = 10, 7
    p = np.sort(rng.uniform(1e2, 1e5, (nv, nlat)), axis=0)[::-1]
    f = rng.standard_normal((nv, nlat))
    targets = np.geomspace(2e5, 10.0, 25)
    a, b = climate.to_pressure_levels(f, p, targets), cl.to_pressure_levels(f, p, targets)
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_allclose(a[~np.isnan(a)], b[~np.isnan(b)], rtol=1e-12, atol=1e-14)
