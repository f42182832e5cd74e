"""Energy fixer and budget of the CUDA path (through the C ABI) against the
oracle (oracle/energy.py): float64 mode within 1e-10 relative per field,
budget rows to round-off, the fixer's dT within the spread that the state's
own round-off leaves in a difference of two nearly equal energies."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from harness import Pair, field_errors
from oracle import diagnostics as dg
from oracle import dycore as dc
import workloads as wls

SMALL = wls.HS_G4.with_(name="hs_g3_L12", glevel=3, nv=12, n_large=3)


@pytest.mark.parametrize("forcing,graph", [("held_suarez", False), ("none", True)])
def test_fixer_and_budget_match_the_oracle(forcing, graph):
    wl = SMALL.with_(forcing=forcing)
    st = torch.cuda.Stream() if graph else None
    p = Pair(wl, stream=st.cuda_stream if st is not None else None)
    try:
        thor.thor_tune(p.state, thor.THOR_TUNE_ENERGY_FIXER, 1)
        thor.thor_tune(p.state, thor.THOR_TUNE_BUDGET, 8)
        X = p.oracle_initial()
        budget = []
        ref = dc.run(p.model, X, wl.n_large, wl.n_small, wl.dt, energy_fixer=True, budget=budget)
        thor.thor_step(p.state, wl.n_large, wl.n_small, wl.dt)
        e = field_errors(p.get(), ref)
        assert e["rho"] < 1e-10 and e["Th"] < 1e-10 and e["M"] < 1e-10 and e["W"] < 1e-10, e
        rows = thor.thor_budget_read(p.state)
        budget = np.array(budget)
        assert rows.shape == budget.shape == (wl.n_large, 8)
        np.testing.assert_allclose(rows[:, :6], budget[:, :6], rtol=1e-12, atol=0)
        assert np.all(np.sign(rows[:, 6]) == np.sign(budget[:, 6])) and np.all(budget[:, 6] != 0)
        np.testing.assert_allclose(rows[:, 6], budget[:, 6], rtol=0.05, atol=0)
    finally:
        p.close()


def test_fixer_keeps_total_energy_without_forcing():
    """Float64, no forcing: with the fixer the total energy of thor_diag after
    three large steps equals the initial one to round-off; without it the
    dynamics change it measurably."""
    wl = SMALL.with_(forcing="none")
    drift = {}
    for fix in (0, 1):
        p = Pair(wl)
        try:
            thor.thor_tune(p.state, thor.THOR_TUNE_ENERGY_FIXER, fix)
            e0 = thor.thor_diag(p.state)["energy"]
            thor.thor_step(p.state, wl.n_large, wl.n_small, wl.dt)
            drift[fix] = abs(thor.thor_diag(p.state)["energy"] - e0) / e0
        finally:
            p.close()
    assert drift[0] > 1e-11, drift
    assert drift[1] < 1e-13, drift


def test_budget_rows_chain_with_the_state_diagnostics():
    """Each row's start values are thor_diag of the state before that large
    step; the dynamics conserve mass; recording stops at the capacity."""
    wl = SMALL
    p = Pair(wl)
    try:
        thor.thor_tune(p.state, thor.THOR_TUNE_BUDGET, 2)
        diags = []
        for _ in range(3):
            diags.append(thor.thor_diag(p.state))
            thor.thor_step(p.state, 1, wl.n_small, wl.dt)
        rows = thor.thor_budget_read(p.state)
        assert rows.shape == (2, 8)
        for r, d in zip(rows, diags):
            assert r[0] == pytest.approx(d["mass"], rel=1e-15)
            assert r[1] == pytest.approx(d["energy"], rel=1e-15)
            assert r[2] == pytest.approx(d["aam"], rel=1e-15)
            assert abs(r[3] - r[0]) <= 1e-13 * r[0]
            assert r[6] == 0.0                     # fixer off
        thor.thor_tune(p.state, thor.THOR_TUNE_BUDGET, 0)
        assert thor.thor_budget_read(p.state).shape == (0, 8)
    finally:
        p.close()


def test_mixed_precision_fixer_runs_and_records():
    """Float32 storage: the fixer's correction (about 1e-9 of the energy) is
    near the storage's resolution, so only the record and finiteness are
    checked, and that the energy stays within 1e-6 of its start."""
    wl = SMALL.with_(forcing="none")
    p = Pair(wl, precision=thor.THOR_MIXED)
    try:
        thor.thor_tune(p.state, thor.THOR_TUNE_ENERGY_FIXER, 1)
        thor.thor_tune(p.state, thor.THOR_TUNE_BUDGET, 4)
        e0 = thor.thor_diag(p.state)["energy"]
        thor.thor_step(p.state, wl.n_large, wl.n_small, wl.dt)
        d = thor.thor_diag(p.state)
        rows = thor.thor_budget_read(p.state)
        assert d["nonfinite"] == 0 and rows.shape == (wl.n_large, 8)
        assert abs(d["energy"] - e0) <= 1e-6 * e0
        assert np.all(np.isfinite(rows))
    finally:
        p.close()
