"""Oracle global diagnostics, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3 calls dry mass "a robust invariant" of the flux-form equations and
discusses total energy and axial angular momentum as the quantities whose
numerical sources need watching (Sec. 3, Sec. 6.1). The cell volume is
A_c r_k^2 dz_k (deep atmosphere).
"""

import numpy as np

from . import dycore as dc
from . import operators as op


def volumes(model):
    return model.grid.area[:, None] * model.vg.rc[None, :] ** 2 * model.vg.dz[None, :]


def diagnostics(model, X):
    pl, vg = model.planet, model.vg
    V = volumes(model)
    p = dc.pressure(pl, X.Th)
    T = dc.temperature(pl, X.rho, p)
    Wc = op.interp_to_centres(vg, X.W)
    rhat = model.rhat
    mom = X.M + Wc[..., None] * rhat[:, None, :]
    ke = 0.5 * np.sum(mom ** 2, axis=-1) / X.rho
    energy = np.sum(V * (X.rho * pl.cv * T + ke + X.rho * pl.gravity * vg.zc[None, :]))
    r = vg.rc[None, :, None] * rhat[:, None, :]
    ang = r[..., 0] * mom[..., 1] - r[..., 1] * mom[..., 0]
    planet_ang = X.rho * pl.omega * (r[..., 0] ** 2 + r[..., 1] ** 2)
    rho_i = op.interp_to_interfaces(vg, X.rho)
    w = X.W[:, 1:-1] / rho_i[:, 1:-1]
    fields = [X.rho, X.M, X.W, X.Th]
    return dict(
        mass=float(np.sum(V * X.rho)),
        energy=float(energy),
        aam=float(np.sum(V * (ang + planet_ang))),
        max_vh=float(np.max(np.linalg.norm(X.M / X.rho[..., None], axis=-1))),
        max_w=float(np.max(np.abs(w))) if w.size else 0.0,
        mean_T=float(np.sum(V * T) / np.sum(V)),
        nonfinite=int(sum(np.count_nonzero(~np.isfinite(f)) for f in fields)),
    )
