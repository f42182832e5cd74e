"""The benchmark size (glevel 6 x 32 levels, 40962 columns): one float64
large step against the oracle's, and properties that hold at any size,
checked in the launch configuration bench.py times (float32 mixed with the
TMA-staged column solve and the autotuned launch shape, float64, graph
replay)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from harness import Pair, change_errors, field_errors, init_struct, moving_start, planet_struct
from oracle import dycore as dc
import workloads as wls

WL = wls.HS_G6


def _grid():
    P = WL.planet
    return thor.thor_grid_create(WL.glevel, WL.nv, P.radius, WL.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, WL.spring_max_iter))


def _state(grid, wl, precision, stream):
    return thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, precision), stream)


@pytest.fixture(scope="module")
def grid():
    g = _grid()
    yield g
    thor.thor_grid_destroy(g)


@pytest.mark.parametrize("precision, tol", [(thor.THOR_FP64, 1e-12), (thor.THOR_MIXED, 1e-12)])
def test_mass_conserved_full_size(grid, precision, tol):
    s = torch.cuda.Stream()
    st = _state(grid, WL, precision, s.cuda_stream)
    try:
        m0 = thor.thor_diag(st)["mass"]
        thor.thor_step(st, 3, WL.n_small, WL.dt)
        d = thor.thor_diag(st)
        assert d["nonfinite"] == 0
        assert abs(d["mass"] - m0) / m0 < (tol if precision == thor.THOR_FP64 else 1e-7)
    finally:
        thor.thor_state_destroy(st)


@pytest.mark.parametrize("precision, vmax", [(thor.THOR_FP64, 1e-8), (thor.THOR_MIXED, 1e-3)])
def test_rest_full_size(grid, precision, vmax):
    wl = WL.with_(forcing="none", noise_amp=0.0)
    s = torch.cuda.Stream()
    st = _state(grid, wl, precision, s.cuda_stream)
    try:
        thor.thor_step(st, 3, wl.n_small, wl.dt)
        d = thor.thor_diag(st)
        assert d["max_vh"] < vmax and d["max_w"] < vmax, d
    finally:
        thor.thor_state_destroy(st)


@pytest.mark.slow
def test_fp64_large_step_matches_oracle_full_size():
    """One large step (3 slow-term evaluations, 13 small steps, Held-Suarez
    physics) of the float64 path at 40962 x 32 against the oracle's, every
    field to 1e-10 relative; the oracle needs about a minute for it."""
    wl = WL.with_(n_large=1)
    p = Pair(wl, precision=thor.THOR_FP64)
    try:
        X = p.oracle_initial()
        ref = dc.large_step(p.model, X, wl.dt, wl.n_small)
        thor.thor_step(p.state, 1, wl.n_small, wl.dt)
        got = p.get()
        e = field_errors(got, ref)
        assert max(e["rho"], e["Th"], e["M"], e["W"]) < 1e-10, e
        c = change_errors(got, ref, X)
        assert max(c.values()) < 1e-8, c
    finally:
        p.close()


def test_fp64_first_small_step_matches_oracle_full_size():
    """The first RK stage alone (one slow-term evaluation and one small step
    of dt/3, THOR_TUNE_RK_STAGES = 1) at 40962 x 32 in float64 against the
    oracle's rk_stage, from a moving start: every field to 1e-10 relative L2
    and every element to 1e-8 of its field's largest change."""
    wl = WL.with_(n_large=1)
    p = Pair(wl, precision=thor.THOR_FP64)
    try:
        X = moving_start(p, p.oracle_initial())
        ref = dc.rk_stage(p.model, X, X, wl.dt / 3.0, 1, p.model.Kd(wl.dt))
        thor.thor_tune(p.state, thor.THOR_TUNE_RK_STAGES, 1)
        thor.thor_step(p.state, 1, wl.n_small, wl.dt)
        got = p.get()
        e = field_errors(got, ref)
        assert max(e["rho"], e["Th"], e["M"], e["W"]) < 1e-10, e
        c = change_errors(got, ref, X)
        assert max(c.values()) < 1e-8, c
    finally:
        p.close()


@pytest.mark.slow
def test_fp64_hot_jupiter_large_step_matches_oracle_full_size():
    """The hot-Jupiter workload at full size (40962 x 32, R = 1e8 m, 220 bar
    to 1 mbar, dt 300 s, 6 small steps, Newtonian relaxation to the day-night
    T_eq of Sec. 6.2 with the seeded contrast): one float64 large step
    against the oracle's, every field to 1e-10 relative L2, from a moving
    start (from rest the dynamics of the first step leave M at zero, where
    the oracle keeps float64 rounding noise; the heating acts at its end)."""
    wl = wls.HJ_G6.with_(n_large=1)
    p = Pair(wl, precision=thor.THOR_FP64)
    try:
        X = moving_start(p, p.oracle_initial(), amp=50.0)
        ref = dc.large_step(p.model, X, wl.dt, wl.n_small)
        thor.thor_step(p.state, 1, wl.n_small, wl.dt)
        got = p.get()
        e = field_errors(got, ref)
        w_scale = wl.planet.gravity * float(np.max(ref.rho)) * wl.dt / wl.n_small
        assert max(e["rho"], e["Th"], e["M"]) < 1e-10, e
        assert e["W"] < 1e-10 or e["W_maxabs"] < 1e-12 * w_scale, e
    finally:
        p.close()


def test_mixed_tracks_fp64_full_size(grid):
    """Three large steps of the float32 path, with the launch shape the
    autotuner picks (as bench.py runs it), stay within the mixed-mode
    tolerances of the float64 path at full size."""
    s = torch.cuda.Stream()
    out = []
    for prec in (thor.THOR_FP64, thor.THOR_MIXED):
        st = _state(grid, WL, prec, s.cuda_stream)
        try:
            if prec == thor.THOR_MIXED:
                thor.thor_autotune(st, WL.n_small, WL.dt, steps=1)
            thor.thor_step(st, 3, WL.n_small, WL.dt)
            out.append({f: thor.thor_state_get(st, f, WL.ncol, WL.nv)
                        for f in (thor.THOR_FIELD_RHO, thor.THOR_FIELD_TEMPERATURE, thor.THOR_FIELD_MOM)})
        finally:
            thor.thor_state_destroy(st)
    a, b = out
    rel = lambda f: np.linalg.norm(b[f] - a[f]) / np.linalg.norm(a[f])
    assert rel(thor.THOR_FIELD_RHO) < 1e-6
    assert rel(thor.THOR_FIELD_TEMPERATURE) < 1e-6
    assert rel(thor.THOR_FIELD_MOM) < 1e-2


def test_graph_matches_direct_full_size(grid):
    s = torch.cuda.Stream()
    res = []
    for graph in (1, 0):
        st = _state(grid, WL, thor.THOR_MIXED, s.cuda_stream)
        try:
            thor.thor_tune(st, thor.THOR_TUNE_GRAPH, graph)
            thor.thor_step(st, 2, WL.n_small, WL.dt)
            res.append(thor.thor_state_get(st, thor.THOR_FIELD_MOM, WL.ncol, WL.nv))
        finally:
            thor.thor_state_destroy(st)
    assert np.array_equal(res[0], res[1])
