"""Pins of the oracle dynamical core (Sec. 3-4) against invariants, closed
forms and the discrete equations it solves. CPU only."""

import numpy as np
import pytest

from conftest import oracle_grid
from oracle import diagnostics as dg
from oracle import dycore as dc
from oracle import operators as op
from oracle.grid import lonlat
import workloads as wls


def _model(glevel=3, nv=10, z_top=30.0e3, forcing="none", **kw):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    G = oracle_grid(glevel, max_iter=10, tol=0.0)
    return dc.Model(G, op.VerticalGrid(nv, z_top, P.radius), pl, forcing=forcing, **kw)


def _smooth_u(m):
    lon, lat = lonlat(m.grid.points)
    return 0.5 + 0.5 * np.cos(lat)[:, None] * np.cos(lon)[:, None] * \
        np.sin(np.pi * m.vg.zc / m.vg.zi[-1])[None, :]


def test_equation_of_state_round_trip():
    """Eq. pressure with the ideal gas gives theta = T (p_ref/p)^(Rd/cp)."""
    m = _model()
    pl = m.planet
    rho = np.array([1.2, 0.3, 1e-3])
    T = np.array([300.0, 220.0, 180.0])
    p = rho * pl.Rd * T
    Th = dc.rhotheta_from_p(pl, p)
    assert np.allclose(dc.pressure(pl, Th), p, rtol=1e-14)
    assert np.allclose(Th / rho, T * (pl.p_ref / p) ** (pl.Rd / pl.cp), rtol=1e-14)


def test_small_step_satisfies_discrete_equations():
    """After one small step the four unsubstituted discrete relations (Eqs.
    dens2, pt2, momr2 and the linear pressure advance of the vertical solve)
    hold, checked with the operators alone, not the assembled matrix."""
    m = _model(glevel=2, nv=8)
    vg, pl = m.vg, m.planet
    u = _smooth_u(m)
    X = dc.initial_state(m, 290.0, 1.0e5, 2.0, u)
    rng = np.random.default_rng(3)
    X.M[:] = op.project_h(m.rhat, rng.standard_normal(X.M.shape))
    X.W[:, 1:-1] = 0.01 * rng.standard_normal((X.W.shape[0], vg.nv - 1))
    Kd = m.Kd(1800.0)
    co = dc.slow_terms(m, X, Kd)
    pert = dict(rho=1e-4 * rng.standard_normal(X.rho.shape), M=np.zeros_like(X.M),
                W=np.zeros_like(X.W), Th=X.Th * (1 + 1e-5 * rng.standard_normal(X.Th.shape)))
    pert["p"] = dc.pressure(pl, pert["Th"]) - co["p"]
    dtau = 300.0
    new = dc.small_step(m, X, co, pert, dtau, Kd)
    p_lin = pert["p"] + co["Pi"] * (new["Th"] - pert["Th"])
    rho_i = op.interp_to_interfaces(vg, new["rho"])
    W_expect = pert["W"] + dtau * (co["S_W"] - op.ddz_at_interfaces(vg, p_lin) - pl.gravity * rho_i)
    W_expect[:, [0, -1]] = 0.0
    scale = np.abs(new["W"]).max()
    assert np.max(np.abs(new["W"] - W_expect)) < 1e-10 * scale
    assert np.all(new["W"][:, [0, -1]] == 0.0)
    rho_expect = pert["rho"] + dtau * (co["S_rho"] - op.div_h_levels(m.grid, vg, new["M"])
                                       - op.div_v(vg, new["W"]))
    assert np.max(np.abs(new["rho"] - rho_expect)) < 1e-12 * np.abs(X.rho).max()
    Wtot = X.W + new["W"]
    Th_expect = pert["Th"] + dtau * (co["S_Th"]
                                     - op.div_h_levels(m.grid, vg, co["theta"][..., None] * (X.M + new["M"]))
                                     - op.div_v(vg, co["theta_i"] * Wtot))
    assert np.max(np.abs(new["Th"] - Th_expect)) < 1e-12 * np.abs(X.Th).max()
    assert np.allclose(new["p"], dc.pressure(pl, new["Th"]) - co["p"], rtol=0,
                       atol=1e-9 * co["p"].max())


def test_vertical_system_is_tridiagonal_and_matches_dense():
    """The assembled vertical operator couples only neighbouring interfaces."""
    m = _model(glevel=1, nv=7)
    Dv, Gz, Iz = dc.vertical_matrices(m.vg)
    rng = np.random.default_rng(0)
    th = 300 + rng.random(m.vg.nv - 1)
    Pi = 1.4 * (1 + 0.1 * rng.random(m.vg.nv))
    A = np.eye(m.vg.nv - 1) - 90000.0 * (Gz * Pi[None, :]) @ (Dv * th[None, :]) \
        - 90000.0 * 9.8 * Iz @ Dv
    band = np.abs(np.subtract.outer(np.arange(m.vg.nv - 1), np.arange(m.vg.nv - 1))) > 1
    assert np.all(A[band] == 0.0)


def test_rest_state_stays_at_rest():
    """An isothermal atmosphere at rest in discrete hydrostatic balance, no
    forcing and no noise: |v| < 1e-8 m/s after 10 large steps."""
    m = _model(glevel=3, nv=20, z_top=36.0e3)
    X = dc.initial_state(m, 300.0, 1.0e5)
    X = dc.run(m, X, 10, 6, 1800.0)
    d = dg.diagnostics(m, X)
    assert d["max_vh"] < 1e-8 and d["max_w"] < 1e-8


def test_mass_conserved_with_forcing():
    """Flux form (Sec. 3): global mass is conserved to round-off, with the
    Held-Suarez forcing and noise on."""
    m = _model(glevel=3, nv=10, forcing="held_suarez")
    X = dc.initial_state(m, 300.0, 1.0e5, 0.1, np.random.default_rng(7).random((m.grid.ncol, 10)))
    m0 = dg.diagnostics(m, X)["mass"]
    X = dc.run(m, X, 10, 6, 1800.0)
    d = dg.diagnostics(m, X)
    assert abs(d["mass"] - m0) / m0 < 1e-12
    assert d["max_vh"] > 1e-3          # the forcing did move the air


def test_uniform_theta_stays_uniform():
    """With Eq. pt2 read as the flux of the same total momentum as Eq. dens2,
    rho theta = theta0 rho is preserved exactly (hyperdiffusion and physics
    off, which alone act on theta)."""
    m = _model(glevel=3, nv=6, z_top=3.0e3, hyperdiffusion=False)
    u = _smooth_u(m)
    X = dc.initial_state(m, 300.0, 1.0e5, 3.0, u)
    theta0 = float(np.mean(X.Th / X.rho))
    X.Th[:] = theta0 * X.rho
    X = dc.run(m, X, 3, 6, 600.0)
    th = X.Th / X.rho
    assert np.max(np.abs(th - theta0)) < 1e-10 * theta0
    assert dg.diagnostics(m, X)["max_vh"] > 1e-3


def test_time_step_consistency():
    """Self-convergence in dt at a fixed end time with fixed K_d. The fast
    vertical terms are backward Euler (Eq. momr2 at tau + dtau), so the
    momentum errors fall at first order: the ratio of successive differences
    is about 2. A sign or index slip in a slow term stops the convergence."""
    m = _model(glevel=2, nv=8, z_top=20.0e3, Kd_fixed=1e14)
    X0 = dc.initial_state(m, 300.0, 1.0e5, 1.0, _smooth_u(m))
    runs = {dt: dc.run(m, X0, int(round(3600.0 / dt)), 6, dt) for dt in (1200.0, 600.0, 300.0)}
    for f in ("M", "W"):
        e1 = np.linalg.norm(getattr(runs[1200.0], f) - getattr(runs[600.0], f))
        e2 = np.linalg.norm(getattr(runs[600.0], f) - getattr(runs[300.0], f))
        assert 1.6 < e1 / e2 < 2.6, (f, e1 / e2)


def test_hyperdiffusion_of_a_harmonic():
    """Eq. diff_rho on rho = rho0 (1 + eps Y_2): F_rho = -K_d (6/r^2)^2 (rho - rho0)
    at every level, four rings away from the pentagons, on the converged
    modified grid. (Applied twice, the Sec. 4 Laplacian amplifies its own
    grid-scale error, so the agreement is a few percent, not second order.)"""
    P_ = wls.EARTH
    pl = dc.Planet(P_.radius, P_.omega, P_.gravity, P_.Rd, P_.cp, P_.p_ref,
                   dc.diffusion_parameter(P_.dt_paper, P_.tau_d))
    m = dc.Model(oracle_grid(3), op.VerticalGrid(3, 30.0e3, P_.radius), pl)
    P = m.grid.points
    Y = P[:, 0] * P[:, 1]
    rho0 = 1.1
    X = dc.State(rho0 * (1 + 1e-3 * Y)[:, None] * np.ones(3), np.zeros((m.grid.ncol, 3, 3)),
                 np.zeros((m.grid.ncol, 4)), np.full((m.grid.ncol, 3), 330.0))
    Kd = 1.0e16
    F_rho, F_M, F_W, F_Th = dc.hyperdiffusion(m, X, dc.pressure(m.planet, X.Th), Kd)
    exact = -Kd * (6.0 / m.vg.rc[None, :] ** 2) ** 2 * (X.rho - rho0)
    near = set(np.where(m.grid.nn == 5)[0].tolist())
    for _ in range(4):
        for i in list(near):
            near.update(m.grid.nbr[i, :m.grid.nn[i]].tolist())
    mask = np.ones(m.grid.ncol, bool)
    mask[list(near)] = False
    rel = np.linalg.norm((F_rho - exact)[mask]) / np.linalg.norm(exact[mask])
    assert rel < 0.05
    assert np.all(F_M == 0.0) and np.all(F_W == 0.0)


def test_stage_schedule():
    """Sec. 3: 1 small step of dt/3, n/2 of dt/n, n of dt/n."""
    s = dc.stage_schedule(600.0, 8)
    assert s == [(200.0, 1), (75.0, 4), (75.0, 8)]
    with pytest.raises(ValueError):
        dc.stage_schedule(600.0, 7)


def test_diffusion_parameter_reproduces_tau_d():
    """Eqs. kd and tau_d: with D = dt/(32 tau_d), K_d = D dbar^4/dt gives back
    tau_d = dbar^4/(32 K_d) at any resolution."""
    import json, os
    t1 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "forcing_constants.json")))["table1"]
    for key in ("earth", "hot_jupiter"):
        e = t1[key]
        D = dc.diffusion_parameter(e["dt"], e["tau_d"])
        for g in (4, 5, 6):
            dbar = np.sqrt(2 * np.pi / 5) * e["radius"] / 2 ** g
            Kd = D * dbar ** 4 / e["dt"]
            assert dbar ** 4 / (32 * Kd) == pytest.approx(e["tau_d"], rel=1e-14)


def _rest_model(omega, hyper=False, glevel=3, nv=4):
    P_ = wls.EARTH
    pl = dc.Planet(P_.radius, omega, P_.gravity, P_.Rd, P_.cp, P_.p_ref,
                   dc.diffusion_parameter(P_.dt_paper, P_.tau_d))
    return dc.Model(oracle_grid(glevel), op.VerticalGrid(nv, 8.0e3, P_.radius), pl,
                    hyperdiffusion=hyper)


def test_coriolis_term():
    """Eq. mom: the Coriolis force -2 Omega x (rho v). For a tiny horizontal
    momentum on a resting, balanced column, S_M = -(2 Omega z x M)_h and
    S_W = -(2 Omega z x M)_r at the interfaces, up to O(M^2) advection."""
    m = _rest_model(7.292e-5)
    X = dc.initial_state(m, 280.0, 1.0e5)
    rng = np.random.default_rng(2)
    M = op.project_h(m.rhat, rng.standard_normal((m.grid.ncol, 1, 3))) * np.ones((1, 4, 1))
    X.M[:] = 1e-4 * M
    co = dc.slow_terms(m, X, 0.0)
    cor = 2.0 * np.cross(np.array([0, 0, 7.292e-5])[None, None, :], X.M)
    scale = np.abs(cor).max()
    assert np.max(np.abs(co["S_M"] + op.project_h(m.rhat, cor))) < 1e-5 * scale
    cr = op.interp_to_interfaces(m.vg, op.radial(m.rhat, cor))
    assert np.max(np.abs(co["S_W"][:, 1:-1] + cr[:, 1:-1])) < 1e-5 * scale


def test_advection_of_solid_body_rotation():
    """Eq. mom advection div(rho v v) for v = w z x r at uniform density is the
    centripetal -rho w^2 (x, y, 0) r: its horizontal part enters -S_M and its
    radial part -S_W (pressure balanced, Omega = 0, no diffusion)."""
    m = _rest_model(0.0)
    X = dc.initial_state(m, 280.0, 1.0e5)
    w = 2.0e-5
    R = m.vg.rc[None, :, None] * m.rhat[:, None, :]
    v = w * np.cross(np.array([0, 0, 1.0])[None, None, :], R)
    X.M[:] = X.rho[..., None] * v
    co = dc.slow_terms(m, X, 0.0)
    acc = -X.rho[..., None] * w ** 2 * R * np.array([1.0, 1.0, 0.0])
    exact_h = op.project_h(m.rhat, acc)
    rel = np.linalg.norm(-co["S_M"] - exact_h) / np.linalg.norm(exact_h)
    assert rel < 0.02, rel
    ar = op.interp_to_interfaces(m.vg, op.radial(m.rhat, acc))[:, 1:-1]
    rel_r = np.linalg.norm(-co["S_W"][:, 1:-1] - ar) / np.linalg.norm(ar)
    assert rel_r < 0.02, rel_r


def test_pressure_gradient_force():
    """Eq. mom2 slow term -grad_h p / r: with p = p_bal(z)(1 + eps z/|r|) and
    M = 0, S_M = -eps p_bal grad_h(z)/r (no advection, no Coriolis)."""
    m = _rest_model(0.0)
    X = dc.initial_state(m, 280.0, 1.0e5)
    pl = m.planet
    p = dc.pressure(pl, X.Th)
    Y = m.rhat[:, 2]
    p2 = p * (1.0 + 1e-4 * Y[:, None])
    X.Th[:] = dc.rhotheta_from_p(pl, p2)
    co = dc.slow_terms(m, X, 0.0)
    gradY = op.project_h(m.rhat, np.broadcast_to(np.array([0, 0, 1.0]), (m.grid.ncol, 3)).copy())
    exact = -1e-4 * p[..., None] * gradY[:, None, :] / m.vg.rc[None, :, None]
    rel = np.linalg.norm(co["S_M"] - exact) / np.linalg.norm(exact)
    assert rel < 0.01, rel


def test_divergence_damping_dissipates_divergence():
    """Eqs. diff_vx-vz divergence damping lowers the area-weighted squared
    3-D divergence of the momentum (K_d > 0 damps)."""
    m = _rest_model(0.0, glevel=3, nv=4)
    X = dc.initial_state(m, 280.0, 1.0e5)
    rng = np.random.default_rng(4)
    M = op.project_h(m.rhat, rng.standard_normal(X.M.shape))
    g, vg = m.grid, m.vg
    D0 = op.div_h_levels(g, vg, M)
    G = op.grad_h_levels(g, vg, D0)
    Kd = 0.2 * m.Kd(1800.0)
    M1 = M + 100.0 * op.project_h(m.rhat, -Kd * op.vlap_levels(g, vg, G))
    D1 = op.div_h_levels(g, vg, M1)
    w = g.area[:, None]
    assert np.sum(w * D1 ** 2) < np.sum(w * D0 ** 2)


def test_pressure_hyperdiffusion_enters_rho_theta():
    """Eq. diff_p converted to rho theta (reading R4): for T = T0 (1 + eps Y_2)
    at uniform rho, F_Th = Th/(gamma p) (-Rd rho K_d lap lap T), with
    lap lap Y_2 = 36 Y_2 / r^4 (four rings from the pentagons)."""
    m = _rest_model(0.0, hyper=True)
    pl = m.planet
    P = m.grid.points
    Y = P[:, 0] * P[:, 1]
    N = m.grid.ncol
    rho = np.full((N, 4), 1.1)
    T = 290.0 * (1 + 1e-3 * Y)[:, None] * np.ones(4)
    X = dc.State(rho, np.zeros((N, 4, 3)), np.zeros((N, 5)), dc.rhotheta_from_p(pl, rho * pl.Rd * T))
    p = dc.pressure(pl, X.Th)
    Kd = 1.0e16
    _, _, _, F_Th = dc.hyperdiffusion(m, X, p, Kd)
    exact = X.Th / (pl.gamma * p) * (-pl.Rd * rho * Kd * 36.0 / m.vg.rc[None, :] ** 4 * (T - 290.0))
    near = set(np.where(m.grid.nn == 5)[0].tolist())
    for _ in range(4):
        for i in list(near):
            near.update(m.grid.nbr[i, :m.grid.nn[i]].tolist())
    mask = np.ones(N, bool)
    mask[list(near)] = False
    assert np.linalg.norm((F_Th - exact)[mask]) / np.linalg.norm(exact[mask]) < 0.05


def test_diagnostics_closed_forms():
    """Mass and axial angular momentum of uniform-density air at rest on a
    rotating planet against the shell integrals: M = rho (4 pi/3)(r1^3 - r0^3),
    AAM = rho Omega (8 pi/15)(r1^5 - r0^5)."""
    m = _rest_model(7.292e-5, glevel=3, nv=8)
    N = m.grid.ncol
    X = dc.State(np.full((N, 8), 1.3), np.zeros((N, 8, 3)), np.zeros((N, 9)), np.full((N, 8), 400.0))
    d = dg.diagnostics(m, X)
    r0, r1 = m.vg.ri[0], m.vg.ri[-1]
    assert d["mass"] == pytest.approx(1.3 * 4 * np.pi / 3 * (r1 ** 3 - r0 ** 3), rel=1e-7)
    assert d["aam"] == pytest.approx(1.3 * 7.292e-5 * 8 * np.pi / 15 * (r1 ** 5 - r0 ** 5), rel=1e-2)
    assert d["max_vh"] == 0.0 and d["nonfinite"] == 0
