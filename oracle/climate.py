"""Oracle zonal band means of one state, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 6.1 judges the Held-Suarez climate by zonal and time averages: the
eastward and northward wind, temperature, the mass stream function built
from the averaged northward wind (Eq. for Psi), and the eddy fluxes
[u'v'] and [v'T'] with phi' = phi - (zonal mean of phi). Reading C-1: on the
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
the ideal gas.
"""

import numpy as np

from . import dycore as dc
from .diagnostics import volumes
from .grid import lonlat

QUANTITIES = ("weight", "u", "v", "T", "p", "uv", "vT", "uu", "vv")


def band_of(points, nlat):
    """Latitude band of every column (reading C-1)."""
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
