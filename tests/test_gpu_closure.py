"""Learned closure: trained on the GPU by the library's own kernels on
Held-Suarez glevel-6 runs coarse-grained to glevel 5 (32 levels), judged
against the coarse-grained glevel-6 truth and the plain glevel-5 method."""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from conftest import report_dir
from paper_1607_05535_gb300 import closure as cl
import workloads as wls


def test_coarse_grain_of_rest_is_rest_and_conserves_mass():
    """Area-weighted coarse graining maps the balanced resting state onto the
    coarse grid's own balanced resting state (same reference column)."""
    wl = wls.HS_G4.with_(noise_amp=0.0, forcing="none")
    su = cl.make_setup(wl, 4, 3, thor.THOR_FP64, None)
    thor.thor_coarse_grain(su.fine, su.coarse, su.fmap)
    a = cl.column_fields(su.coarse, su.ncol_c, su.nv)
    b = cl.column_fields(su.scratch, su.ncol_c, su.nv)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_coarse_grain_and_features_match_host():
    """thor_coarse_grain equals the area-weighted mean over each coarse
    column's fine members (momentum projected onto the coarse tangent plane,
    W zero at the boundaries), and thor_closure_features equals the column's
    deviations from the reference column and its neighbour-mean anomalies,
    both recomputed here on the host from the fine state and the grid tables."""
    wl = wls.HS_G4
    su = cl.make_setup(wl, 4, 3, thor.THOR_FP64, None)
    try:
        thor.thor_step(su.fine, 3, wl.n_small, wl.dt)
        nv, ncf, ncc = su.nv, su.ncol_f, su.ncol_c
        rest_init = thor.thor_init(wl.T0, wl.p_surf, 0.0, wl.seed, 1, wl.hj_dT, thor.THOR_FP64, 1, 1)
        rest = thor.thor_state_init(su.coarse_grid, cl_planet(wl), rest_init, None)
        ref = cl.column_fields(rest, ncc, nv)[0]               # the resting state is the reference column
        thor.thor_state_destroy(rest)
        thor.thor_coarse_grain(su.fine, su.coarse, su.fmap)
        F = cl.column_fields(su.fine, ncf, nv)
        Wf = thor.thor_state_get(su.fine, thor.THOR_FIELD_W, ncf, nv)
        area = thor.thor_grid_areas(su.fine_grid)
        w = np.zeros(ncc)
        np.add.at(w, su.fmap, area)
        E = np.zeros((ncc, 5 * nv))
        np.add.at(E, su.fmap, F * area[:, None])
        E /= w[:, None]
        EW = np.zeros((ncc, nv + 1))
        np.add.at(EW, su.fmap, Wf * area[:, None])
        EW /= w[:, None]
        EW[:, 0] = EW[:, nv] = 0.0
        r = thor.thor_grid_points(su.coarse_grid)
        r /= np.linalg.norm(r, axis=1, keepdims=True)
        m = np.stack([E[:, nv:2 * nv], E[:, 2 * nv:3 * nv], E[:, 3 * nv:4 * nv]], axis=-1)
        m -= np.einsum("ckd,cd->ck", m, r)[..., None] * r[:, None, :]
        E[:, nv:2 * nv], E[:, 2 * nv:3 * nv], E[:, 3 * nv:4 * nv] = m[..., 0], m[..., 1], m[..., 2]
        got = cl.column_fields(su.coarse, ncc, nv)
        for f in range(5):
            sl = slice(f * nv, (f + 1) * nv)
            d = got[:, sl] - E[:, sl]
            scale = np.max(np.abs(E[:, sl] - (ref[sl] if f in (0, 4) else 0.0))) + 1e-300
            assert np.max(np.abs(d)) <= 1e-10 * scale, (f, np.max(np.abs(d)) / scale)
        gW = thor.thor_state_get(su.coarse, thor.THOR_FIELD_W, ncc, nv)
        assert np.max(np.abs(gW - EW)) <= 1e-10 * (np.max(np.abs(EW)) + 1e-300)

        x = cl.features(su.coarse, ncc, nv, torch, "cuda").double().cpu().numpy()
        dev = got - np.where(np.isin(np.arange(5 * nv) // nv, [0, 4]), ref, 0.0)
        nbr = thor.thor_grid_neighbours(su.coarse_grid)
        anom = np.empty_like(dev)
        for c in range(ncc):
            q = [j for j in nbr[c] if j >= 0 and j != c]
            anom[c] = dev[q].mean(axis=0) - dev[c]
        for blk, want in ((slice(0, 5 * nv), dev), (slice(5 * nv, 10 * nv), anom)):
            scale = np.max(np.abs(want), axis=0) + 1e-300
            assert np.all(np.abs(x[:, blk] - want) <= 1e-5 * scale + 1e-30)
    finally:
        cl.destroy_setup(su)


def test_closure_window_semantics():
    """With a window of n large steps, the closure's state after n steps is
    the plain state after n steps plus n dt tau_hat(features of the start
    state), momentum correction projected onto the tangent plane."""
    wl = wls.HS_G4.with_(dt=900.0)
    torch.cuda.set_device(0)
    su = cl.make_setup(wl, 4, 3, thor.THOR_FP64, None)
    ncol, nv, n = su.ncol_c, su.nv, 3
    net = thor.thor_mlp_create([10 * nv, 64, 5 * nv], 256, seed=5)
    try:
        dev = "cuda"
        x0 = torch.empty((ncol, 10 * nv), dtype=torch.float32, device=dev)
        thor.thor_closure_features(su.coarse, torch.zeros(10 * nv, device=dev), torch.ones(10 * nv, device=dev), x0)
        xm, xs = x0.mean(0), x0.std(0).clamp_min(1e-6)
        ym = torch.zeros(5 * nv, device=dev)
        ys = torch.full((5 * nv,), 1e-8, device=dev)
        xn = ((x0 - xm) / xs).contiguous()
        y = cl.predict(net, xn, 5 * nv, 256, torch)
        tau = (y * ys + ym).double().cpu().numpy()
        rhat = thor.thor_grid_points(su.coarse_grid)
        rhat = rhat / np.linalg.norm(rhat, axis=1, keepdims=True)
        m = np.stack([tau[:, nv:2 * nv], tau[:, 2 * nv:3 * nv], tau[:, 3 * nv:4 * nv]], axis=-1)
        m -= np.einsum("ckd,cd->ck", m, rhat)[..., None] * rhat[:, None, :]
        tau[:, nv:2 * nv], tau[:, 2 * nv:3 * nv], tau[:, 3 * nv:4 * nv] = m[..., 0], m[..., 1], m[..., 2]

        thor.thor_closure_attach(su.coarse, net, xm.contiguous(), xs.contiguous(), ym, ys, period=n)
        thor.thor_step(su.coarse, n - 1, wl.n_small, wl.dt)      # the window spans two calls
        thor.thor_step(su.coarse, 1, wl.n_small, wl.dt)
        thor.thor_closure_attach(su.coarse, None)
        thor.thor_step(su.scratch, n, wl.n_small, wl.dt)
        d = cl.column_fields(su.coarse, ncol, nv) - cl.column_fields(su.scratch, ncol, nv)
        want = n * wl.dt * tau
        assert np.max(np.abs(want)) > 0
        np.testing.assert_allclose(d, want, rtol=0, atol=1e-5 * np.max(np.abs(want)))
    finally:
        thor.thor_mlp_destroy(net)


def test_closure_gain_over_plain_coarse_method():
    """A priori: the n-step residual tendency predicted on held-out windows.
    A posteriori: four windows of coarse large steps with the closure (after
    three rounds of dataset aggregation) against the coarse-grained fine run,
    compared with the plain coarse method, from two held-out starts."""
    wl = wls.HS_G6
    dev = "cuda"
    torch.cuda.set_device(0)
    su = cl.make_setup(wl, 6, 5, thor.THOR_MIXED, None)
    ncol, nv, window = su.ncol_c, su.nv, 4
    cl.spin_up(su, wl, 600)
    X, Y = cl.generate_samples(su, wl, 24, torch, dev, window=window)
    Xtr, Ytr = torch.cat(X[:20]), torch.cat(Y[:20])
    Xte, Yte = torch.cat(X[20:]), torch.cat(Y[20:])
    del X, Y
    xm, xs, ym, ys = cl.normalisation(Xtr, Ytr, torch)
    net0 = thor.thor_mlp_create([10 * nv, 256, 256, 256, 5 * nv], 1024, seed=11)
    try:
        hist = cl.train(net0, ((Xtr - xm) / xs).contiguous(), ((Ytr - ym) / ys).contiguous(), epochs=20,
                        batch=1024, lr=1e-3, torch=torch)
        P = cl.predict(net0, ((Xte - xm) / xs).contiguous(), 5 * nv, 1024, torch) * ys + ym
    finally:
        thor.thor_mlp_destroy(net0)
    err_closure = float(((P - Yte) ** 2).mean())
    err_plain = float((Yte ** 2).mean())              # the plain coarse method adds no correction
    gain = 1.0 - err_closure / err_plain
    report = {"samples_train": int(Xtr.shape[0]), "samples_test": int(Xte.shape[0]), "loss_history": hist,
              "tendency_mse_closure": err_closure, "tendency_mse_plain": err_plain, "a_priori_gain": gain}
    del Xtr, Ytr, Xte, Yte, P

    net, norm, hists = cl.fit(su, wl, torch, dev, windows=24, window=window, rounds=3)
    try:
        runs = []
        for _ in range(2):
            runs.append(cl.rollout_errors(su, wl, net, norm, window, 4))
            thor.thor_step(su.fine, 8, wl.n_small, wl.dt)
    finally:
        thor.thor_mlp_destroy(net)
    cl.destroy_setup(su)
    e_c = np.mean([r[0] for r in runs], axis=0)
    e_p = np.mean([r[1] for r in runs], axis=0)
    report.update({"aggregation_loss_history": hists, "rollout_window": window,
                   "rollout_rmse_closure": e_c.tolist(), "rollout_rmse_plain": e_p.tolist(),
                   "rollouts": runs, "a_posteriori_gain": float(1.0 - e_c.mean() / e_p.mean())})
    out = report_dir()
    if out:
        json.dump(report, open(os.path.join(out, "closure_report.json"), "w"), indent=1)
    print({k: v for k, v in report.items() if "history" not in k})
    assert hist[-1] < hist[0]
    assert gain > 0.25, report
    assert np.all(e_c < e_p), report


def cl_planet(wl):
    P = wl.planet
    return thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)


def cl_init(wl):
    return thor.thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, 1, wl.hj_dT, thor.THOR_MIXED, 1, 1)
