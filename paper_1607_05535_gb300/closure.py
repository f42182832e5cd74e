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
the coarse state of the column and its neighbour-mean anomalies. Online the
closure (thor_closure_attach with period n) evaluates tau_hat at the start of
each window and adds n dt tau_hat at its end, so that one window reproduces
the target's definition.

A network trained only on coarse-grained fine states sees, from the second
window on, states that the coarse model and the closure produced, and its
errors compound. Dataset aggregation closes that gap: further samples start
from closure-corrected coarse runs of the previous network (generate_samples
with ``net``), and the next network trains on the union.
"""

from dataclasses import dataclass

import numpy as np

from . import (THOR_FIELD_MOM, THOR_FIELD_RHO, THOR_FIELD_RHOTHETA, thor_closure_attach, thor_grid_coarse_map,
               thor_closure_features, thor_coarse_grain, thor_grid_create, thor_grid_info,
               thor_grid_points, thor_init, thor_mlp_forward, thor_mlp_train_step, thor_planet,
               thor_grid_destroy, thor_mlp_create, thor_mlp_destroy, thor_spring, thor_state_destroy,
               thor_state_get, thor_state_init, thor_state_set, thor_step)

FIELDS = 5


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
    extra: object             # a third coarse state (closure runs)
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
    extra = thor_state_init(gc, planet, init, stream)
    # coarse column whose centre is nearest to each fine centre (the coarse
    # control volume containing it, up to the centroid offsets)
    fmap = thor_grid_coarse_map(gf, gc)
    return Setup(gf, gc, fine, coarse, scratch, extra, fmap, thor_grid_info(gf)["ncol"],
                 thor_grid_info(gc)["ncol"], wl.nv)


def destroy_setup(su):
    for st in (su.fine, su.coarse, su.scratch, su.extra):
        thor_state_destroy(st)
    thor_grid_destroy(su.fine_grid)
    thor_grid_destroy(su.coarse_grid)


def spin_up(su, wl, steps):
    thor_step(su.fine, steps, wl.n_small, wl.dt)


def _set_fields(state, A, nv):
    thor_state_set(state, THOR_FIELD_RHO, np.ascontiguousarray(A[:, :nv]))
    mom = np.stack([A[:, nv:2 * nv], A[:, 2 * nv:3 * nv], A[:, 3 * nv:4 * nv]], axis=-1)
    thor_state_set(state, THOR_FIELD_MOM, np.ascontiguousarray(mom))
    thor_state_set(state, THOR_FIELD_RHOTHETA, np.ascontiguousarray(A[:, 4 * nv:]))


def _project(tau, rhat, nv):
    """Momentum part of a (ncol, 5 nv) tendency projected onto the tangent
    plane, as the closure applies it."""
    t = tau.copy()
    m = np.stack([t[:, nv:2 * nv], t[:, 2 * nv:3 * nv], t[:, 3 * nv:4 * nv]], axis=-1)
    m -= np.einsum("ckd,cd->ck", m, rhat)[..., None] * rhat[:, None, :]
    t[:, nv:2 * nv], t[:, 2 * nv:3 * nv], t[:, 3 * nv:4 * nv] = m[..., 0], m[..., 1], m[..., 2]
    return t


def features(state, ncol, nv, torch, device):
    """Raw (unnormalised) closure features of a state, [ncol, 10 nv] float32."""
    x = torch.empty((ncol, 2 * FIELDS * nv), dtype=torch.float32, device=device)
    z = torch.zeros(2 * FIELDS * nv, dtype=torch.float32, device=device)
    thor_closure_features(state, z, z + 1.0, x)
    return x


def tendency(net, norm, state, ncol, nv, torch, device):
    """tau_hat of a state as a (ncol, 5 nv) float64 host array."""
    xm, xs, ym, ys = norm
    x = ((features(state, ncol, nv, torch, device) - xm) / xs).contiguous()
    return (predict(net, x, FIELDS * nv, 1024, torch) * ys + ym).double().cpu().numpy()


def generate_samples(su, wl, windows, torch, device, window=4, net=None, norm=None, chain=3):
    """Samples over `windows` consecutive windows of n = `window` large steps
    of the fine run. Plain samples: features of C(X_f(t)), target
    [C(X_f(t + n dt)) - S_c^n(C(X_f(t)))] / (n dt). With a trained network,
    chained samples as well (dataset aggregation, Ross, Gordon and Bagnell
    2011): a coarse run restarted from C(X_f) every `chain` windows and
    corrected by the network at each window's end, so that later windows
    start from states the closure itself produces online; their target is
    the same n-step residual from that state (the chain runs in su.extra).
    Returns feature and target lists of [ncol, .] float32 device tensors."""
    nv, ncol, n = su.nv, su.ncol_c, window
    extra = su.extra
    Xs, Ys = [], []
    rhat = None
    if net is not None:
        rhat = thor_grid_points(su.coarse_grid)
        rhat = rhat / np.linalg.norm(rhat, axis=1, keepdims=True)
    for w in range(windows):
        thor_coarse_grain(su.fine, su.scratch, su.fmap)                 # C(X_f(t))
        Xs.append(features(su.scratch, ncol, nv, torch, device))
        thor_step(su.scratch, n, wl.n_small, wl.dt)                     # S_c^n(C(X_f(t)))
        plain = column_fields(su.scratch, ncol, nv)
        if net is not None:
            if w % chain == 0:
                thor_coarse_grain(su.fine, extra, su.fmap)
            else:
                Xs.append(features(extra, ncol, nv, torch, device))
            tau = _project(tendency(net, norm, extra, ncol, nv, torch, device), rhat, nv)
            thor_step(extra, n, wl.n_small, wl.dt)
            chained = column_fields(extra, ncol, nv)
        thor_step(su.fine, n, wl.n_small, wl.dt)
        thor_coarse_grain(su.fine, su.coarse, su.fmap)                  # C(X_f(t + n dt))
        truth = column_fields(su.coarse, ncol, nv)
        Ys.append(torch.tensor((truth - plain) / (n * wl.dt), dtype=torch.float32, device=device))
        if net is not None:
            if w % chain != 0:
                Ys.append(torch.tensor((truth - chained) / (n * wl.dt), dtype=torch.float32, device=device))
            _set_fields(extra, chained + n * wl.dt * tau, nv)
    return Xs, Ys


def rollout_errors(su, wl, net, norm, window, windows):
    """From the current coarse-grained fine state, `windows` windows of
    coarse large steps with the closure attached (period = window) and
    without, against the coarse-grained fine run. Returns two lists (closure,
    plain) of normalised RMS errors at each window's end: every (field,
    level) scaled by its standard deviation over the columns of the truth."""
    ncol, nv = su.ncol_c, su.nv
    xm, xs, ym, ys = norm
    extra = su.extra
    thor_coarse_grain(su.fine, extra, su.fmap)
    thor_coarse_grain(su.fine, su.scratch, su.fmap)
    thor_closure_attach(extra, net, xm, xs, ym, ys, period=window)
    e_c, e_p = [], []
    try:
        for _ in range(windows):
            thor_step(extra, window, wl.n_small, wl.dt)
            thor_step(su.scratch, window, wl.n_small, wl.dt)
            thor_step(su.fine, window, wl.n_small, wl.dt)
            thor_coarse_grain(su.fine, su.coarse, su.fmap)
            truth = column_fields(su.coarse, ncol, nv)
            scale = np.std(truth, axis=0) + 1e-30
            e_c.append(float(np.sqrt(np.mean(((column_fields(extra, ncol, nv) - truth) / scale) ** 2))))
            e_p.append(float(np.sqrt(np.mean(((column_fields(su.scratch, ncol, nv) - truth) / scale) ** 2))))
    finally:
        thor_closure_attach(extra, None)
    return e_c, e_p


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


def fit(su, wl, torch, device, windows=24, window=4, rounds=2, chains=(3, 4), epochs=(20, 12, 8),
        hidden=(256, 256, 256), batch=1024, lr=1e-3, seed=11):
    """Trains the closure from the current fine state: plain samples over
    `windows` windows, then `rounds` rounds of dataset aggregation, each a
    fresh network trained on the union of every sample so far. The last
    network is returned with its normalisation and, per round, the loss
    history; the caller destroys the network (thor_mlp_destroy)."""
    nv = su.nv
    sizes = [2 * FIELDS * nv, *hidden, FIELDS * nv]
    X, Y = generate_samples(su, wl, windows, torch, device, window=window)
    net, norm, hists = None, None, []
    for r in range(rounds + 1):
        if r > 0:
            Xr, Yr = generate_samples(su, wl, windows, torch, device, window=window, net=net, norm=norm,
                                      chain=chains[min(r - 1, len(chains) - 1)])
            X, Y = X + Xr, Y + Yr
            thor_mlp_destroy(net)
        Xa, Ya = torch.cat(X), torch.cat(Y)
        norm = normalisation(Xa, Ya, torch)
        xm, xs, ym, ys = norm
        net = thor_mlp_create(sizes, batch, seed=seed)
        hists.append(train(net, ((Xa - xm) / xs).contiguous(), ((Ya - ym) / ys).contiguous(),
                           epochs=epochs[min(r, len(epochs) - 1)], batch=batch, lr=lr, torch=torch))
        del Xa, Ya
    return net, norm, hists
