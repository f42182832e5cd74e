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


def test_closure_gain_over_plain_coarse_method():
    wl = wls.HS_G6
    dev = "cuda"
    torch.cuda.set_device(0)
    su = cl.make_setup(wl, 6, 5, thor.THOR_MIXED, None)
    n_train, n_test = 20, 4
    X, Y = cl.generate_samples(su, wl, spinup=600, snapshots=n_train + n_test, spacing=2, torch=torch,
                               device=dev, window=4)
    ncol, nv = su.ncol_c, su.nv
    ntr = n_train * ncol
    xm, xs, ym, ys = cl.normalisation(X[:ntr], Y[:ntr], torch)
    Xn = ((X - xm) / xs).contiguous()
    Yn = ((Y - ym) / ys).contiguous()
    net = thor.thor_mlp_create([10 * nv, 256, 256, 256, 5 * nv], 1024, seed=11)
    try:
        hist = cl.train(net, Xn[:ntr], Yn[:ntr], epochs=20, batch=1024, lr=1e-3, torch=torch)
        P = cl.predict(net, Xn[ntr:], 5 * nv, 1024, torch) * ys + ym
        Yt = Y[ntr:]
        err_closure = float(((P - Yt) ** 2).mean())
        err_plain = float((Yt ** 2).mean())          # the plain coarse method adds no correction
        gain = 1.0 - err_closure / err_plain
        report = {"samples_train": ntr, "samples_test": n_test * ncol, "loss_history": hist,
                  "tendency_mse_closure": err_closure, "tendency_mse_plain": err_plain,
                  "a_priori_gain": gain}

        # a posteriori: from a held-out coarse-grained state, 8 coarse large
        # steps with the closure (evaluated every 4 steps, its training
        # window) and without, against the coarse-grained fine run
        thor.thor_coarse_grain(su.fine, su.coarse, su.fmap)
        thor.thor_coarse_grain(su.fine, su.scratch, su.fmap)
        thor.thor_closure_attach(su.coarse, net, xm, xs, ym, ys, period=4)
        thor.thor_step(su.coarse, 8, wl.n_small, wl.dt)
        thor.thor_closure_attach(su.coarse, None)
        thor.thor_step(su.scratch, 8, wl.n_small, wl.dt)
        thor.thor_step(su.fine, 8, wl.n_small, wl.dt)
        truth_state = thor.thor_state_init(su.coarse_grid, cl_planet(wl), cl_init(wl), None)
        thor.thor_coarse_grain(su.fine, truth_state, su.fmap)
        truth = cl.column_fields(truth_state, ncol, nv)
        thor.thor_state_destroy(truth_state)
        with_c = cl.column_fields(su.coarse, ncol, nv)
        plain = cl.column_fields(su.scratch, ncol, nv)
        scale = np.std(truth, axis=0) + 1e-30
        e_c = float(np.sqrt(np.mean(((with_c - truth) / scale) ** 2)))
        e_p = float(np.sqrt(np.mean(((plain - truth) / scale) ** 2)))
        report.update({"rollout_steps": 8, "rollout_rmse_closure": e_c, "rollout_rmse_plain": e_p})
    finally:
        thor.thor_mlp_destroy(net)
    out = os.path.join(os.path.dirname(os.path.dirname(__file__)), "gpurun_out")
    if os.path.isdir(out):
        json.dump(report, open(os.path.join(out, "closure_report.json"), "w"), indent=1)
    print(report)
    assert hist[-1] < hist[0]
    assert gain > 0.25, report
    assert e_c < e_p, report


def cl_planet(wl):
    P = wl.planet
    return thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)


def cl_init(wl):
    return thor.thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, 1, wl.hj_dT, thor.THOR_MIXED, 1, 1)
