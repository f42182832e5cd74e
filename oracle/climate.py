"""Oracle zonal band means of one state, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 6.1 judges the Held-Suarez climate by zonal and time averages: the
eastward and northward wind, temperature, the mass stream function built
from the averaged northward wind (Eq. for Psi), and the eddy fluxes
[u'v'] and [v'T'] with phi' = phi - (zonal mean of phi). Reading Z-1: on the
icosahedral grid a zonal mean is the volume-weighted mean over the cells of
one level whose latitude falls in one of nlat equal latitude bands (band
b = floor((lat + pi/2 + 1e-9) / pi * nlat), the north pole in the last band;
the 1e-9 rad puts a cell that sits on a band edge, such as the grid's
equatorial cells, in the band north of it whatever the last bits of its
coordinates); the
eddy terms are the band covariances [ab] - [a][b] of one state, averaged in
time by the caller. u and v are the eastward and northward components of
M / rho (the horizontal velocity; both taken as 0 at the two polar cells,
where east and north are undefined), T and p follow from Eq. pressure and
the ideal gas. Reading Z-5 (the grid-imprinting map [w*]) is at w_star;
reading Z-6: pressure-level values come from the time- and zonal-mean
fields on model levels, interpolated in p between the two levels whose
band-mean pressures bracket the target (the paper interpolates each output
before averaging).
"""

import numpy as np

from . import dycore as dc
from .diagnostics import volumes
from .grid import lonlat

QUANTITIES = ("weight", "u", "v", "T", "p", "uv", "vT", "uu", "vv")


def band_of(points, nlat):
    """Latitude band of every column (reading Z-1)."""
    _, lat = lonlat(points)
    return np.minimum(np.floor((lat + 0.5 * np.pi + 1e-9) / np.pi * nlat).astype(int), nlat - 1)


def zonal_band_means(model, X, nlat):
    """(nv, nlat, 9) array: per level and band the total cell volume, the
    volume-weighted means of u, v, T, p and the covariances u'v', v'T',
    u'u', v'v' (zero where a band holds no cell)."""
    pl, pts = model.planet, model.grid.points
    lon, lat = lonlat(pts)
    east = np.stack([-np.sin(lon), np.cos(lon), np.zeros_like(lon)], axis=-1)
    north = np.stack([-np.sin(lat) * np.cos(lon), -np.sin(lat) * np.sin(lon), np.cos(lat)], axis=-1)
    polar = np.hypot(pts[:, 0], pts[:, 1]) < 1e-9
    east[polar] = 0.0
    north[polar] = 0.0
    vel = X.M / X.rho[..., None]
    u = np.einsum("ckj,cj->ck", vel, east)
    v = np.einsum("ckj,cj->ck", vel, north)
    p = dc.pressure(pl, X.Th)
    T = dc.temperature(pl, X.rho, p)
    V = volumes(model)
    band = band_of(pts, nlat)
    nv = model.vg.nv
    out = np.zeros((nv, nlat, 9))
    for k in range(nv):
        w = V[:, k]
        W = np.bincount(band, weights=w, minlength=nlat)
        mean = lambda f: np.divide(np.bincount(band, weights=w * f, minlength=nlat), W,
                                   out=np.zeros(nlat), where=W > 0)
        mu, mv, mT, mp = mean(u[:, k]), mean(v[:, k]), mean(T[:, k]), mean(p[:, k])
        out[k, :, 0] = W
        out[k, :, 1:5] = np.stack([mu, mv, mT, mp], axis=-1)
        out[k, :, 5] = mean(u[:, k] * v[:, k]) - mu * mv
        out[k, :, 6] = mean(v[:, k] * T[:, k]) - mv * mT
        out[k, :, 7] = mean(u[:, k] ** 2) - mu ** 2
        out[k, :, 8] = mean(v[:, k] ** 2) - mv ** 2
    return out


def cell_w(model, X):
    """Vertical velocity at every cell centre, (N, nv): the vertical momentum
    interpolated linearly (Lagrange k = 1, Sec. 2.1) from the interfaces to
    the centre, over the density."""
    from . import operators as op
    return op.interp_to_centres(model.vg, X.W) / X.rho


def w_star(model, w_mean, nlat):
    """The grid-imprinting map of Sec. 6.1 (reading Z-5): the time mean [w]
    of every cell minus the volume-weighted mean of [w] over its latitude
    band at the same level, (N, nv). The paper writes w* = w - [w] with [.]
    the time average and maps [w*]; taken literally that is zero, so the
    deviation is read as the one from the zonal mean (the prime of the eddy
    terms), whose time average keeps what the grid imprints."""
    V = volumes(model)
    band = band_of(model.grid.points, nlat)
    out = np.empty_like(w_mean)
    for k in range(w_mean.shape[1]):
        W = np.bincount(band, weights=V[:, k], minlength=nlat)
        m = np.bincount(band, weights=V[:, k] * w_mean[:, k], minlength=nlat)
        out[:, k] = w_mean[:, k] - np.divide(m, W, out=np.zeros(nlat), where=W > 0)[band]
    return out


def to_pressure_levels(values, p_mean, p_levels):
    """Sec. 6: results shown against pressure are interpolated linearly to a
    pressure grid after the run. values and p_mean (nv, nlat) on model
    levels (p_mean the band's mean pressure, reading Z-6) ->
    (len(p_levels), nlat); a target outside a band's pressure range is NaN."""
    nv, nlat = values.shape
    out = np.full((len(p_levels), nlat), np.nan)
    for b in range(nlat):
        p, f = p_mean[:, b], values[:, b]
        for i, pt in enumerate(p_levels):
            for k in range(nv - 1):
                lo, hi = min(p[k], p[k + 1]), max(p[k], p[k + 1])
                if lo <= pt <= hi:
                    out[i, b] = f[k] if hi == lo else f[k] + (f[k + 1] - f[k]) * (pt - p[k]) / (p[k + 1] - p[k])
                    break
    return out
