"""Mixed precision (float32 fields and stencils, float64 elimination and
reductions) against the float64 oracle, per field, on the glevel-4 x 20-level
Held-Suarez workload. The gates are the stated per-field tolerances of the
mixed mode."""

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
from harness import Pair
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls

# stated tolerances after 10 large steps (relative L2 unless noted)
GATES = {"rho": 1e-6, "T": 1e-6, "vh_abs_max": 2e-3, "vh_rel": 1e-2, "w_abs_max": 5e-5}


def field_report(p, X, ref):
    pl = p.model.planet
    T = dc.temperature(pl, X.rho, dc.pressure(pl, X.Th))
    Tr = dc.temperature(pl, ref.rho, dc.pressure(pl, ref.Th))
    vh = X.M / X.rho[..., None]
    vhr = ref.M / ref.rho[..., None]
    ri = op.interp_to_interfaces(p.model.vg, X.rho)[:, 1:-1]
    rir = op.interp_to_interfaces(p.model.vg, ref.rho)[:, 1:-1]
    w, wr = X.W[:, 1:-1] / ri, ref.W[:, 1:-1] / rir
    return {
        "rho": float(np.linalg.norm(X.rho - ref.rho) / np.linalg.norm(ref.rho)),
        "T": float(np.linalg.norm(T - Tr) / np.linalg.norm(Tr)),
        "vh_abs_max": float(np.abs(vh - vhr).max()),
        "vh_rel": float(np.linalg.norm(vh - vhr) / np.linalg.norm(vhr)),
        "vh_max": float(np.abs(vhr).max()),
        "w_abs_max": float(np.abs(w - wr).max()),
        "w_max": float(np.abs(wr).max()),
    }


def test_mixed_vs_oracle_held_suarez_g4():
    wl = wls.HS_G4
    p = Pair(wl, precision=thor.THOR_MIXED)
    try:
        X0 = p.oracle_initial()
        ref = dc.run(p.model, X0, wl.n_large, wl.n_small, wl.dt)
        thor.thor_step(p.state, wl.n_large, wl.n_small, wl.dt)
        rep = field_report(p, p.get(), ref)
    finally:
        p.close()
    out = report_dir()
    if out:
        json.dump(rep, open(os.path.join(out, "mixed_errors_g4.json"), "w"), indent=1)
    print(rep)
    for k, g in GATES.items():
        assert rep[k] < g, (k, rep)


@pytest.mark.parametrize("graph", [False, True])
def test_staged_solve_matches_direct_solve(graph):
    """The TMA-staged column solve (default for float storage) computes the
    same numbers as the direct-load solve: same operations in the same order,
    only the loads differ."""
    import torch
    from harness import init_struct, planet_struct
    wl = wls.HS_G4.with_(n_large=4)
    st = torch.cuda.Stream() if graph else None
    sp = st.cuda_stream if st is not None else None
    grid = thor.thor_grid_create(wl.glevel, wl.nv, wl.planet.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, wl.spring_max_iter))
    a = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, thor.THOR_MIXED), sp)
    b = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, thor.THOR_MIXED), sp)
    try:
        thor.thor_tune(b, thor.THOR_TUNE_SOLVE_TMA, 0)
        for s_ in (a, b):
            thor.thor_step(s_, wl.n_large, wl.n_small, wl.dt)
        for f in (thor.THOR_FIELD_RHO, thor.THOR_FIELD_MOM, thor.THOR_FIELD_W, thor.THOR_FIELD_RHOTHETA):
            x = thor.thor_state_get(a, f, wl.ncol, wl.nv)
            y = thor.thor_state_get(b, f, wl.ncol, wl.nv)
            assert np.array_equal(x, y), f
        assert thor.thor_diag(a)["nonfinite"] == 0
    finally:
        thor.thor_state_destroy(a)
        thor.thor_state_destroy(b)
        thor.thor_grid_destroy(grid)


def test_l2_hints_change_no_value():
    """The L2 eviction priorities of the small steps (THOR_TUNE_L2_HINTS)
    only place lines in the cache: every mode steps a mixed state to the
    same bits; values outside 0..3 are refused."""
    from harness import init_struct, planet_struct
    wl = wls.HS_G4.with_(n_large=3)
    grid = thor.thor_grid_create(wl.glevel, wl.nv, wl.planet.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, wl.spring_max_iter))
    fields = (thor.THOR_FIELD_RHO, thor.THOR_FIELD_MOM, thor.THOR_FIELD_W, thor.THOR_FIELD_RHOTHETA)
    out = []
    try:
        for mode in (0, 1, 2, 3):          # ends at the default, 3
            s_ = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, thor.THOR_MIXED), None)
            try:
                thor.thor_tune(s_, thor.THOR_TUNE_L2_HINTS, mode)
                thor.thor_step(s_, wl.n_large, wl.n_small, wl.dt)
                out.append([thor.thor_state_get(s_, f, wl.ncol, wl.nv) for f in fields])
                with pytest.raises(thor.ThorError):
                    thor.thor_tune(s_, thor.THOR_TUNE_L2_HINTS, 4)
            finally:
                thor.thor_state_destroy(s_)
    finally:
        thor.thor_grid_destroy(grid)
    for o in out[1:]:
        for x, y, f in zip(out[0], o, fields):
            assert np.array_equal(x, y), f


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_level_split_matches_one_chain(prec):
    """The small steps' stencils split into a lower and an upper level half
    on two streams (THOR_TUNE_LEVEL_SPLIT, graph replay) compute the same
    numbers as one chain over all levels."""
    import torch
    from harness import init_struct, planet_struct
    wl = wls.HS_G4.with_(n_large=3)
    p = thor.THOR_MIXED if prec == "mixed" else thor.THOR_FP64
    st = torch.cuda.Stream()
    grid = thor.thor_grid_create(wl.glevel, wl.nv, wl.planet.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, wl.spring_max_iter))
    fields = (thor.THOR_FIELD_RHO, thor.THOR_FIELD_MOM, thor.THOR_FIELD_W, thor.THOR_FIELD_RHOTHETA)
    out = []
    try:
        for split, kc in ((0, 2), (1, 2), (1, 3)):
            s_ = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, p), st.cuda_stream)
            try:
                thor.thor_tune(s_, thor.THOR_TUNE_KCHUNK, kc)
                thor.thor_tune(s_, thor.THOR_TUNE_LEVEL_SPLIT, split)
                thor.thor_step(s_, wl.n_large, wl.n_small, wl.dt)
                out.append([thor.thor_state_get(s_, f, wl.ncol, wl.nv) for f in fields])
            finally:
                thor.thor_state_destroy(s_)
    finally:
        thor.thor_grid_destroy(grid)
    for o in out[1:]:
        for x, y, f in zip(out[0], o, fields):
            assert np.array_equal(x, y), f
