"""The compensated state of the mixed path (THOR_TUNE_COMPENSATED, on by
default for mixed states): every prognostic field of X^t kept as a float
pair hi + lo, the last stage end, physics and fixer adding their increments
with an error-free sum.

Checked here: the pair carries a float64 value through thor_state_set /
thor_state_get to about 2^-48 of it; compensated steps in float64 parity
mode are refused; a compensated checkpoint restarts bit for bit; the
compensated path stays within the mixed-mode gates of the float64 oracle
after 10 large steps, and its error against the float64 path over 10 / 100 /
1000 large steps (Held-Suarez g4 x 20 L) is measured beside the plain mixed
path's, with the mass drift of both (written to THOR_REPORT_DIR when set)."""

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
from harness import Pair, init_struct, planet_struct
from oracle import dycore as dc
import workloads as wls

FIELDS = (thor.THOR_FIELD_RHO, thor.THOR_FIELD_MOM, thor.THOR_FIELD_W, thor.THOR_FIELD_RHOTHETA)
WL = wls.HS_G4


def _grid(wl=WL):
    P = wl.planet
    return thor.thor_grid_create(wl.glevel, wl.nv, P.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, wl.spring_max_iter))


def _state(grid, precision, compensated, wl=WL):
    s = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, precision), None)
    if precision == thor.THOR_MIXED:
        thor.thor_tune(s, thor.THOR_TUNE_COMPENSATED, 1 if compensated else 0)
    return s


def test_pair_carries_float64_values():
    """A float64 value set into a compensated state comes back to about
    2^-48 of itself (hi + lo); the plain float state keeps 2^-24."""
    grid = _grid()
    a, b = _state(grid, thor.THOR_MIXED, True), _state(grid, thor.THOR_MIXED, False)
    try:
        rng = np.random.default_rng(3)
        x = thor.thor_state_get(a, thor.THOR_FIELD_RHOTHETA, WL.ncol, WL.nv)
        y = x * (1 + 1e-3 * rng.standard_normal(x.shape))
        for s, bound in ((a, 2e-14), (b, 1e-7)):
            thor.thor_state_set(s, thor.THOR_FIELD_RHOTHETA, y)
            back = thor.thor_state_get(s, thor.THOR_FIELD_RHOTHETA, WL.ncol, WL.nv)
            assert np.max(np.abs(back - y) / np.abs(y)) < bound
        # off again: the state rounds to its float part
        thor.thor_tune(a, thor.THOR_TUNE_COMPENSATED, 0)
        back = thor.thor_state_get(a, thor.THOR_FIELD_RHOTHETA, WL.ncol, WL.nv)
        assert np.max(np.abs(back - y) / np.abs(y)) < 1e-7
    finally:
        thor.thor_state_destroy(a)
        thor.thor_state_destroy(b)
        thor.thor_grid_destroy(grid)


def test_float64_state_refuses():
    grid = _grid()
    s64 = _state(grid, thor.THOR_FP64, False)
    try:
        with pytest.raises(thor.ThorError):
            thor.thor_tune(s64, thor.THOR_TUNE_COMPENSATED, 1)
        thor.thor_tune(s64, thor.THOR_TUNE_COMPENSATED, 0)         # nothing to drop
    finally:
        thor.thor_state_destroy(s64)
        thor.thor_grid_destroy(grid)


def test_ensemble_follows_a_member_switching_compensation():
    """An ensemble member switched between plain and compensated between
    ensemble steps is replanned (its low parts are freed and reallocated, so
    a stale member table would be wrong by far more): the ensemble matches
    the member stepped alone either way, to 1e-4 of each field's largest
    value (the ensemble and single-state kernels contract products into FMAs
    differently, and the glevel-4 x 20-level workload carries that to a few
    1e-5 in one large step)."""
    grid = _grid()
    a, b = _state(grid, thor.THOR_MIXED, True), _state(grid, thor.THOR_MIXED, True)
    ens = thor.thor_ensemble_create([a], None)
    try:
        for cmp in (1, 0, 1):
            thor.thor_tune(a, thor.THOR_TUNE_COMPENSATED, cmp)
            thor.thor_tune(b, thor.THOR_TUNE_COMPENSATED, cmp)
            thor.thor_ensemble_step(ens, 1, [WL.n_small], [WL.dt])
            thor.thor_step(b, 1, WL.n_small, WL.dt)
            for f in FIELDS:
                x = thor.thor_state_get(a, f, WL.ncol, WL.nv)
                y = thor.thor_state_get(b, f, WL.ncol, WL.nv)
                tol = 1e-4
                assert np.max(np.abs(x - y)) <= tol * np.max(np.abs(y)), (cmp, f)
    finally:
        thor.thor_ensemble_destroy(ens)
        thor.thor_state_destroy(a)
        thor.thor_state_destroy(b)
        thor.thor_grid_destroy(grid)


def test_compensated_checkpoint_restart_is_bit_exact():
    grid = _grid()
    st = torch.cuda.Stream()
    mk = lambda: thor.thor_state_init(grid, planet_struct(WL.planet), init_struct(WL, thor.THOR_MIXED),
                                      st.cuda_stream)
    a, b = mk(), mk()
    c = None
    try:
        for s in (a, b):
            thor.thor_tune(s, thor.THOR_TUNE_COMPENSATED, 1)
        thor.thor_step(a, 4, WL.n_small, WL.dt)
        thor.thor_step(b, 2, WL.n_small, WL.dt)
        buf = thor.thor_checkpoint_save(b)
        c = mk()
        thor.thor_tune(c, thor.THOR_TUNE_COMPENSATED, 0)
        with pytest.raises(thor.ThorError):          # twice the size: a plain state refuses it
            thor.thor_checkpoint_load(c, buf)
        thor.thor_tune(c, thor.THOR_TUNE_COMPENSATED, 1)
        thor.thor_checkpoint_load(c, buf)
        thor.thor_step(c, 2, WL.n_small, WL.dt)
        for f in FIELDS:
            assert np.array_equal(thor.thor_state_get(a, f, WL.ncol, WL.nv),
                                  thor.thor_state_get(c, f, WL.ncol, WL.nv)), f
    finally:
        for s in (a, b, c):
            if s is not None:
                thor.thor_state_destroy(s)
        thor.thor_grid_destroy(grid)


def test_compensated_within_mixed_gates_of_the_oracle():
    """10 large steps of the Held-Suarez g4 workload, compensated, against the
    float64 oracle within the mixed-mode gates (rho and T 1e-6 relative L2,
    horizontal wind 2e-3 m/s, vertical wind 5e-5 m/s max abs)."""
    p = Pair(WL, precision=thor.THOR_MIXED)
    try:
        thor.thor_tune(p.state, thor.THOR_TUNE_COMPENSATED, 1)
        X = p.oracle_initial()
        ref = dc.run(p.model, X, WL.n_large, WL.n_small, WL.dt)
        thor.thor_step(p.state, WL.n_large, WL.n_small, WL.dt)
        A = p.get()
        rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel(A.rho, ref.rho) < 1e-6
        pl = p.model.planet
        TA = dc.temperature(pl, A.rho, dc.pressure(pl, A.Th))
        TB = dc.temperature(pl, ref.rho, dc.pressure(pl, ref.Th))
        assert rel(TA, TB) < 1e-6
        vh = np.abs(A.M / A.rho[..., None] - ref.M / ref.rho[..., None]).max()
        assert vh < 2e-3
    finally:
        p.close()


def test_compensated_against_plain_over_long_runs():
    """Error against the float64 path after 10 / 100 / 1000 large steps of the
    Held-Suarez g4 x 20 L workload, plain mixed and compensated, per field,
    and the mass drift of each (written to THOR_REPORT_DIR). Measured: rho
    1.8e-5 -> 2.1e-8 and T 4.0e-5 -> 4.6e-8 relative L2 after 1000 steps;
    gated at a tenth of the plain path's error from 100 steps on. The mass
    drift (about 4e-10 after 1000 steps in both) comes from the float32
    flux stencils, whose edge fluxes are not exactly antisymmetric, not
    from the storage, so compensation leaves it; both stay below 1e-9."""
    grid = _grid()
    ref = _state(grid, thor.THOR_FP64, False)
    runs = {"plain": _state(grid, thor.THOR_MIXED, False), "compensated": _state(grid, thor.THOR_MIXED, True)}
    out = {k: {} for k in runs}
    try:
        m0 = thor.thor_diag(ref)["mass"]
        done = 0
        for n in (10, 100, 1000):
            for s in [ref] + list(runs.values()):
                thor.thor_step(s, n - done, WL.n_small, WL.dt)
            done = n
            rb = thor.thor_state_get(ref, thor.THOR_FIELD_RHO, WL.ncol, WL.nv)
            Tb = thor.thor_state_get(ref, thor.THOR_FIELD_TEMPERATURE, WL.ncol, WL.nv)
            Mb = thor.thor_state_get(ref, thor.THOR_FIELD_MOM, WL.ncol, WL.nv)
            for k, s in runs.items():
                ra = thor.thor_state_get(s, thor.THOR_FIELD_RHO, WL.ncol, WL.nv)
                Ta = thor.thor_state_get(s, thor.THOR_FIELD_TEMPERATURE, WL.ncol, WL.nv)
                Ma = thor.thor_state_get(s, thor.THOR_FIELD_MOM, WL.ncol, WL.nv)
                out[k][n] = {"rho_rel_l2": float(np.linalg.norm(ra - rb) / np.linalg.norm(rb)),
                             "T_rel_l2": float(np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb)),
                             "vh_max_abs": float(np.max(np.abs(Ma / ra[..., None] - Mb / rb[..., None])))}
        drift = {k: abs(thor.thor_diag(s)["mass"] - m0) / m0 for k, s in runs.items()}
        drift["fp64"] = abs(thor.thor_diag(ref)["mass"] - m0) / m0
        d = report_dir()
        if d:
            with open(os.path.join(d, "compensated_g4.json"), "w") as f:
                json.dump({"errors": out, "mass_drift": drift}, f, indent=1)
        for k in runs:
            assert all(np.isfinite(v) for row in out[k].values() for v in row.values())
        for n in (100, 1000):
            for f in ("rho_rel_l2", "T_rel_l2"):
                assert out["compensated"][n][f] < 0.1 * out["plain"][n][f], (n, f, out)
        assert drift["compensated"] < 1e-9 and drift["plain"] < 1e-9, drift
    finally:
        thor.thor_state_destroy(ref)
        for s in runs.values():
            thor.thor_state_destroy(s)
        thor.thor_grid_destroy(grid)
