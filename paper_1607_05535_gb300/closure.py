"""Learned per-column closure: data generation, training and evaluation.

Orchestration only: every numerical step runs in libthor's kernels (the
dynamical core, thor_coarse_grain, thor_closure_features, the BF16 MLP
training and inference). Host code here arranges arrays, builds the
fine-to-coarse column map and computes normalisation statistics.

Targets. For a fine state X_f(t), let C(.) be the area-weighted coarse
graining and S_c the coarse model's large step. The closure target for the
coarse column fields (rho, M, rho theta at all levels) is

    tau(t) = [ C(X_f(t + n dt)) - S_c^n(C(X_f(t))) ] / (n dt),

the mean tendency the coarse model misses over a window of n large steps
(n = 4 by default; a one-step window is dominated by the fast adjustment of
the coarse-grained state, which the column cannot predict). The features are
the coarse state C(X_f(t)) of the column and its neighbour-mean anomalies.
"""

from dataclasses import dataclass

import numpy as np

from . import (THOR_FIELD_MOM, THOR_FIELD_RHO, THOR_FIELD_RHOTHETA, thor_closure_features,
               thor_coarse_grain, thor_grid_create, thor_grid_info, thor_grid_points, thor_init,
               thor_mlp_create, thor_mlp_forward, thor_mlp_train_step, thor_planet, thor_spring,
               thor_state_get, thor_state_init, thor_state_set, thor_step)

FIELDS = 5


def fine_to_coarse_map(fine_points, coarse_points):
    """Coarse column whose centre is nearest to each fine centre (the coarse
    control volume containing it, up to the centroid offsets)."""
    from scipy.spatial import cKDTree
    return cKDTree(coarse_points).query(fine_points)[1].astype(np.int32)


def column_fields(state, ncol, nv):
    """(ncol, 5 nv) float64 host array: rho, M_x, M_y, M_z, rho theta by level."""
    rho = thor_state_get(state, THOR_FIELD_RHO, ncol, nv)
    mom = thor_state_get(state, THOR_FIELD_MOM, ncol, nv)
    th = thor_state_get(state, THOR_FIELD_RHOTHETA, ncol, nv)
    return np.concatenate([rho, mom[..., 0], mom[..., 1], mom[..., 2], th], axis=1)


@dataclass
class Setup:
    fine_grid: object
    coarse_grid: object
    fine: object
    coarse: object
    scratch: object           # a second coarse state
    fmap: np.ndarray
    ncol_f: int
    ncol_c: int
    nv: int


def make_setup(wl, fine_glevel, coarse_glevel, precision, stream, spring_iters=10):
    P = wl.planet
    sp = thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, spring_iters)
    gf = thor_grid_create(fine_glevel, wl.nv, P.radius, wl.z_top, sp)
    gc = thor_grid_create(coarse_glevel, wl.nv, P.radius, wl.z_top, sp)
    planet = thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
    forcing = {"none": 0, "held_suarez": 1, "hot_jupiter": 2}[wl.forcing]
    init = thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, forcing, wl.hj_dT, precision, 1, 1)
    fine = thor_state_init(gf, planet, init, stream)
    coarse = thor_state_init(gc, planet, init, stream)
    scratch = thor_state_init(gc, planet, init, stream)
    fmap = fine_to_coarse_map(thor_grid_points(gf), thor_grid_points(gc))
    return Setup(gf, gc, fine, coarse, scratch, fmap, thor_grid_info(gf)["ncol"],
                 thor_grid_info(gc)["ncol"], wl.nv)


def generate_samples(su, wl, spinup, snapshots, spacing, torch, device, window=4):
    """Features (raw, float32 device tensor [snapshots * ncol_c, 10 nv]) and
    targets (float32 device tensor [.., 5 nv]) from a fine run."""
    nv, ncol = su.nv, su.ncol_c
    zeros = torch.zeros(2 * FIELDS * nv, dtype=torch.float32, device=device)
    ones = torch.ones(2 * FIELDS * nv, dtype=torch.float32, device=device)
    X = torch.empty((snapshots * ncol, 2 * FIELDS * nv), dtype=torch.float32, device=device)
    Y = torch.empty((snapshots * ncol, FIELDS * nv), dtype=torch.float32, device=device)
    thor_step(su.fine, spinup, wl.n_small, wl.dt)
    for s in range(snapshots):
        thor_coarse_grain(su.fine, su.coarse, su.fmap)               # C(X_f(t))
        thor_closure_features(su.coarse, zeros, ones, X[s * ncol:(s + 1) * ncol])
        thor_coarse_grain(su.fine, su.scratch, su.fmap)
        thor_step(su.scratch, window, wl.n_small, wl.dt)             # S_c^n(C(X_f(t)))
        thor_step(su.fine, window, wl.n_small, wl.dt)
        thor_coarse_grain(su.fine, su.coarse, su.fmap)               # C(X_f(t + n dt))
        tgt = (column_fields(su.coarse, ncol, nv) - column_fields(su.scratch, ncol, nv)) / (window * wl.dt)
        Y[s * ncol:(s + 1) * ncol] = torch.tensor(tgt, dtype=torch.float32, device=device)
        if spacing > 0:
            thor_step(su.fine, spacing, wl.n_small, wl.dt)
    return X, Y


def normalisation(X, Y, torch):
    """Per-feature and per-output mean and standard deviation (floored)."""
    xm, xs = X.mean(0), X.std(0)
    ym, ys = Y.mean(0), Y.std(0)
    xs = torch.where(xs > 1e-12 * (xm.abs() + 1.0), xs, torch.ones_like(xs))
    ys = torch.where(ys > 0, ys, torch.ones_like(ys))
    return xm.contiguous(), xs.contiguous(), ym.contiguous(), ys.contiguous()


def train(net, Xn, Yn, epochs, batch, lr, torch, seed=0):
    """Mini-batch Adam on the normalised data; returns the loss history."""
    n = Xn.shape[0]
    gen = torch.Generator(device=Xn.device)
    gen.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=Xn.device)
    hist = []
    for e in range(epochs):
        perm = torch.randperm(n, generator=gen, device=Xn.device)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            thor_mlp_train_step(net, Xn[idx].contiguous(), Yn[idx].contiguous(), lr, loss)
        hist.append(float(loss.item()))
    return hist


def predict(net, Xn, n_out, batch, torch):
    out = torch.empty((Xn.shape[0], n_out), dtype=torch.float32, device=Xn.device)
    for b0 in range(0, Xn.shape[0], batch):
        xb = Xn[b0:b0 + batch].contiguous()
        yb = torch.empty((xb.shape[0], n_out), dtype=torch.float32, device=Xn.device)
        thor_mlp_forward(net, xb, yb)
        out[b0:b0 + xb.shape[0]] = yb
    return out
