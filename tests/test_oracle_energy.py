"""Pins of the oracle's energy fixer and budgets (oracle/energy.py): what
Sec. 3 fixes (a globally uniform adjustment of the internal energy that keeps
the total energy in balance) and what the mathematics fixes (internal energy
is rho c_v T per unit volume), checked with the independent global
diagnostics of oracle/diagnostics.py."""

import numpy as np

from conftest import oracle_grid
from oracle import diagnostics as dg
from oracle import dycore as dc
from oracle import energy as en
from oracle import operators as op
import workloads as wls


def _model(forcing="none"):
    P = wls.EARTH
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    return dc.Model(oracle_grid(3, max_iter=10, tol=0.0), op.VerticalGrid(10, 30.0e3, P.radius), pl,
                    forcing=forcing)


def _dynamics(m, X, dt=1800.0, n_small=6):
    """The three RK3 stages of a large step without physics (forcing none)."""
    return dc.large_step(m, X, dt, n_small)


def _noisy(m):
    return dc.initial_state(m, 300.0, 1.0e5, 0.1, np.random.default_rng(7).random((m.grid.ncol, m.vg.nv)))


def test_fix_restores_total_energy_with_a_uniform_temperature_change():
    m = _model()
    X0 = _noisy(m)
    Xd = _dynamics(m, X0)
    e0, ed = dg.diagnostics(m, X0)["energy"], dg.diagnostics(m, Xd)["energy"]
    assert abs(ed - e0) > 1e-10 * abs(e0)            # the dynamics do not conserve it exactly
    Xf, dT = en.energy_fix(m, X0, Xd)
    assert abs(dg.diagnostics(m, Xf)["energy"] - e0) <= 1e-13 * abs(e0)
    # uniform: the same temperature increment in every cell
    pl = m.planet
    T = lambda X: dc.temperature(pl, X.rho, dc.pressure(pl, X.Th))
    np.testing.assert_allclose(T(Xf) - T(Xd), dT, rtol=0, atol=1e-9)
    # internal energy sum V rho c_v dT equals the energy that was missing
    V = dg.volumes(m)
    assert abs(np.sum(V * Xd.rho) * pl.cv * dT - (e0 - ed)) <= 1e-12 * abs(e0)
    # density and momentum untouched, mass too
    assert np.array_equal(Xf.rho, Xd.rho) and np.array_equal(Xf.M, Xd.M) and np.array_equal(Xf.W, Xd.W)


def test_fix_of_an_unchanged_state_is_the_identity():
    m = _model()
    X = _noisy(m)
    Xf, dT = en.energy_fix(m, X, X)
    assert dT == 0.0
    np.testing.assert_allclose(Xf.Th, X.Th, rtol=1e-15, atol=0)


def test_fix_cools_when_the_dynamics_gained_energy():
    m = _model()
    X0 = _noisy(m)
    # 1 m/s of extra wind along x, projected to the tangent plane: more kinetic energy
    M = X0.M + np.stack([X0.rho, 0 * X0.rho, 0 * X0.rho], axis=-1)
    M = M - np.sum(M * m.rhat[:, None, :], axis=-1)[..., None] * m.rhat[:, None, :]
    X1 = dc.State(X0.rho.copy(), M, X0.W.copy(), X0.Th.copy())
    assert dg.diagnostics(m, X1)["energy"] > dg.diagnostics(m, X0)["energy"]
    _, dT = en.energy_fix(m, X0, X1)
    assert dT < 0


def test_steps_with_the_fixer_keep_total_energy_without_forcing():
    m = _model()
    X0 = _noisy(m)
    e0 = dg.diagnostics(m, X0)["energy"]
    Xp = dc.run(m, X0, 3, 6, 1800.0)
    budget = []
    Xf = dc.run(m, X0, 3, 6, 1800.0, energy_fixer=True, budget=budget)
    assert abs(dg.diagnostics(m, Xp)["energy"] - e0) > 1e-10 * abs(e0)
    assert abs(dg.diagnostics(m, Xf)["energy"] - e0) <= 1e-13 * abs(e0)
    assert len(budget) == 3
    for r in budget:
        assert abs(r[3] - r[0]) <= 1e-13 * r[0]      # the dynamics conserve mass
        assert r[6] != 0.0


def test_budget_rows_chain_and_separate_dynamics_from_physics():
    """With Held-Suarez forcing: each row's start equals the diagnostics of the
    state the previous step returned, and the fixed dynamics leave the
    physics as the only source of energy change."""
    m = _model("held_suarez")
    X = _noisy(m)
    budget, states = [], [X]
    for _ in range(3):
        X = dc.large_step(m, X, 1800.0, 6, energy_fixer=True, budget=budget)
        states.append(X)
    for n, r in enumerate(budget):
        d = dg.diagnostics(m, states[n])
        assert r[0] == d["mass"] and r[1] == d["energy"] and r[2] == d["aam"]
    # the physics after the fix: E(end) - E(start) is the physics' change alone
    from oracle.physics import apply_physics
    Xd = dc.large_step(_model("none"), states[1], 1800.0, 6)   # dynamics only, same grid and planet
    Xf, _ = en.energy_fix(m, states[1], Xd)
    e_phys = dg.diagnostics(m, apply_physics(m, Xf, 1800.0))["energy"] - dg.diagnostics(m, Xf)["energy"]
    assert abs((dg.diagnostics(m, states[2])["energy"] - budget[1][1]) - e_phys) <= 1e-12 * budget[1][1]
