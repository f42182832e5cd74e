"""Pins of the oracle's anelastic switch (Sec. 3, readings A-1..A-6 in
oracle/anelastic.py). CPU only.

* the projection leaves a momentum whose discrete 3-D divergence is zero to
  the float64 resolution of the operator (1e-9 of the divergence it removes:
  the vertical second differences of p' cancel to about 1e-11 of their
  terms on these anisotropic grids), is idempotent, and removes a pure
  gradient field entirely;
* the operator L = D o G annihilates constants and its columns sum to zero
  with the volume weights (discrete Gauss), so the bordered solve is
  consistent;
* a resting column of the reference stays at rest; a warm anomaly gets the
  Ogura-Phillips buoyancy g rho0 theta' / theta0 at its interfaces;
* rho theta is conserved in volume to rounding without forcing or diffusion,
  and rho stays the reference column;
* sound waves are filtered: a density-only perturbation of the compressible
  model launches acoustic motion at once, while in the anelastic model
  (where the state has no density perturbation) the same theta' only
  moves air through its buoyancy, on the slower gravity-wave scale."""

import numpy as np
import pytest

from conftest import oracle_grid
from oracle import anelastic as an
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls


def _model(glevel=2, nv=8, z_top=2.0e4, omega=None, hyper=True, forcing="none"):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega if omega is None else omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    return dc.Model(oracle_grid(glevel, max_iter=10, tol=0.0), op.VerticalGrid(nv, z_top, P.radius), pl,
                    anelastic=True, hyperdiffusion=hyper, forcing=forcing)


def _random_momentum(m, seed):
    rng = np.random.default_rng(seed)
    N, nv = m.grid.ncol, m.vg.nv
    Mh = op.project_h(m.rhat, rng.standard_normal((N, nv, 3)))
    Wh = np.zeros((N, nv + 1))
    Wh[:, 1:-1] = 0.01 * rng.standard_normal((N, nv - 1))
    return Mh, Wh


@pytest.mark.parametrize("glevel", [2, 3])
def test_projection_is_divergence_free_and_idempotent(glevel):
    m = _model(glevel)
    an.anelastic_start(m, 290.0, 1.0e5)
    Mh, Wh = _random_momentum(m, 1)
    M, W, phi = an.project(m, Mh, Wh, 300.0)
    D0 = np.abs(an.divergence(m, Mh, Wh)).max()
    assert np.abs(an.divergence(m, M, W)).max() < 1e-9 * D0
    assert np.all(W[:, 0] == 0.0) and np.all(W[:, -1] == 0.0)
    assert np.abs(op.radial(m.rhat, M)).max() < 1e-14 * np.abs(M).max()
    M2, W2, phi2 = an.project(m, M, W, 300.0)
    assert np.abs(M2 - M).max() < 1e-9 * np.abs(M).max()
    assert np.abs(W2 - W).max() < 1e-9 * np.abs(W).max()
    V = an.volumes(m)
    assert abs(np.sum(V * phi)) < 1e-12 * np.sum(V * np.abs(phi))


def test_projection_removes_a_gradient():
    """M^ = G_h psi, W^ = G_v psi is all gradient: the projection returns zero
    momentum and p' = psi / dt_s up to its volume mean. (At glevel 3 the
    discrete gradient annihilates the constants only; at glevel 2 it has one
    more null mode, which leaves p' undetermined there but not M and W.)"""
    m = _model(3)
    an.anelastic_start(m, 290.0, 1.0e5)
    rng = np.random.default_rng(4)
    psi = rng.standard_normal((m.grid.ncol, m.vg.nv))
    dts = 200.0
    Mh = op.grad_h_levels(m.grid, m.vg, psi)
    Wh = an.grad_v(m.vg, psi)
    M, W, phi = an.project(m, Mh, Wh, dts)
    assert np.abs(M).max() < 1e-8 * np.abs(Mh).max()
    assert np.abs(W).max() < 1e-8 * np.abs(Wh).max()
    V = an.volumes(m)
    ref = psi / dts - np.sum(V * psi / dts) / np.sum(V)
    assert np.abs(phi - ref).max() < 1e-8 * np.abs(ref).max()


def test_operator_null_spaces():
    """L 1 = 0 (the gradient of a constant vanishes, Sec. 2.1) and
    V^T L = 0 (discrete Gauss: the volume sum of any discrete divergence
    vanishes)."""
    m = _model(2)
    L = an.operator(m)
    n = L.shape[0]
    scale = abs(L).max()
    assert np.abs(L @ np.ones(n)).max() < 1e-12 * scale
    v = an.volumes(m).ravel()
    assert np.abs(L.T @ v).max() < 1e-12 * scale * v.max()


def test_rest_stays_at_rest_and_buoyancy_closed_form():
    m = _model(2, omega=7.292e-5)
    X = an.anelastic_start(m, 280.0, 1.0e5)
    Y = dc.run(m, X, 4, 6, 900.0)
    assert np.abs(Y.M).max() < 1e-12 and np.abs(Y.W).max() < 1e-12
    assert np.array_equal(Y.rho, X.rho)
    # a warm anomaly of 1 K in one column: S_W = g rho0_i (theta' / theta0)_i there
    tp = np.zeros((m.grid.ncol, m.vg.nv))
    tp[5, 3] = 1.0
    X = an.anelastic_start(m, 280.0, 1.0e5, theta_prime=tp)
    rho0, theta0 = m.reference
    S_M, S_W, S_Th = an.slow_terms(m, X, 0.0)
    vg = m.vg
    w0 = (vg.zi[3] - vg.zc[3]) / (vg.zc[2] - vg.zc[3])
    w1 = (vg.zi[3] - vg.zc[2]) / (vg.zc[3] - vg.zc[2])
    b3 = m.planet.gravity * (w0 * rho0[2] + w1 * rho0[3]) * (w1 * 1.0 / theta0[3])
    assert S_W[5, 3] == pytest.approx(b3, rel=1e-12)
    assert S_W[5, 4] > 0 and S_W[5, 3] > 0
    assert np.all(S_W[:5] == 0.0)


def test_rho_theta_conserved_and_rho_fixed():
    """Without forcing and diffusion the volume sum of rho theta is conserved
    (flux form, reading A-3) and rho stays the reference column."""
    m = _model(2, hyper=False, omega=7.292e-5)
    rng = np.random.default_rng(6)
    X = an.anelastic_start(m, 280.0, 1.0e5, theta_prime=rng.standard_normal((m.grid.ncol, m.vg.nv)))
    V = an.volumes(m)
    s0 = np.sum(V * X.Th)
    Y = dc.run(m, X, 4, 6, 900.0)
    assert abs(np.sum(V * Y.Th) - s0) < 1e-14 * s0
    assert np.array_equal(Y.rho, X.rho)
    assert np.abs(an.divergence(m, Y.M, Y.W)).max() < 1e-9 * np.abs(Y.M).max() / m.vg.rc[0] * 1e3


def test_sound_waves_filtered():
    """The compressible model answers a density-only perturbation (theta' at
    fixed pressure) with acoustic motion within one small step; the anelastic
    model answers the same theta' only through its buoyancy: after one
    large step of 60 s its vertical momentum is of the size of the buoyancy
    impulse, far below the compressible model's."""
    rng = np.random.default_rng(8)
    P = wls.EARTH
    pl = dc.Planet(P.radius, 0.0, P.gravity, P.Rd, P.cp, P.p_ref, 0.0)
    G = oracle_grid(2, max_iter=10, tol=0.0)
    vg = op.VerticalGrid(8, 2.0e4, P.radius)
    tp = 0.5 * rng.standard_normal((G.ncol, 8))
    mc = dc.Model(G, vg, pl, hyperdiffusion=False, divergence_damping=False)
    ma = dc.Model(G, vg, pl, hyperdiffusion=False, divergence_damping=False, anelastic=True)
    # compressible: theta' at fixed pressure is a density perturbation
    u = (tp / 0.5 + 1.0) / 2.0
    Xc = dc.initial_state(mc, 280.0, 1.0e5, 0.5, np.clip(u, 0.0, 1.0 - 1e-16))
    Xa = an.anelastic_start(ma, 280.0, 1.0e5, theta_prime=tp)
    Yc = dc.large_step(mc, Xc, 60.0, 6)
    Ya = dc.large_step(ma, Xa, 60.0, 6)
    rho0, theta0 = ma.reference
    impulse = P.gravity * rho0.max() * np.abs(tp).max() / theta0.min() * 60.0
    assert np.abs(Ya.W).max() < 2.0 * impulse
    assert np.abs(Yc.W).max() > 5.0 * np.abs(Ya.W).max()
