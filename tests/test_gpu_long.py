"""Longer runs: mixed precision against float64 at 10, 100 and 1000 large
steps (the float64 path itself matches the oracle to 1e-10, test_gpu_parity),
and restart bit-equality through thor_state_get / thor_state_set."""

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
from harness import init_struct, planet_struct
import workloads as wls

FIELDS = (thor.THOR_FIELD_RHO, thor.THOR_FIELD_MOM, thor.THOR_FIELD_W, thor.THOR_FIELD_RHOTHETA)


def _grid(wl):
    return thor.thor_grid_create(wl.glevel, wl.nv, wl.planet.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, wl.spring_max_iter))


def _errors(a, b, wl):
    n, nv = wl.ncol, wl.nv
    g = lambda s, f: thor.thor_state_get(s, f, n, nv)
    rho_a, rho_b = g(a, thor.THOR_FIELD_RHO), g(b, thor.THOR_FIELD_RHO)
    T_a, T_b = g(a, thor.THOR_FIELD_TEMPERATURE), g(b, thor.THOR_FIELD_TEMPERATURE)
    v_a = g(a, thor.THOR_FIELD_MOM) / rho_a[..., None]
    v_b = g(b, thor.THOR_FIELD_MOM) / rho_b[..., None]
    W_a, W_b = g(a, thor.THOR_FIELD_W), g(b, thor.THOR_FIELD_W)
    rl2 = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
    return {"rho_rel_l2": rl2(rho_a, rho_b), "T_rel_l2": rl2(T_a, T_b),
            "vh_rel_l2": rl2(v_a, v_b), "vh_max_abs": float(np.max(np.abs(v_a - v_b))),
            "vh_max": float(np.max(np.abs(v_b))), "W_max_abs": float(np.max(np.abs(W_a - W_b))),
            "W_max": float(np.max(np.abs(W_b)))}


def test_mixed_against_float64_at_10_100_1000_large_steps():
    """Held-Suarez g4 x 20 L (dt 1800 s, 6 small steps) from rest + 0.1 K
    noise. Gates at 10 and 100 steps; at 1000 steps (about 21 days, when the
    baroclinic instability has started to amplify the seeded noise and every
    rounding difference with it) the errors are reported and the mixed run is
    only required to stay finite with its mass conserved like the float64 run."""
    wl = wls.HS_G4
    grid = _grid(wl)
    a = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, thor.THOR_MIXED), None)
    b = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, thor.THOR_FP64), None)
    report = {}
    try:
        m0a, m0b = thor.thor_diag(a)["mass"], thor.thor_diag(b)["mass"]
        done = 0
        for n in (10, 100, 1000):
            thor.thor_step(a, n - done, wl.n_small, wl.dt)
            thor.thor_step(b, n - done, wl.n_small, wl.dt)
            done = n
            e = _errors(a, b, wl)
            da, db = thor.thor_diag(a), thor.thor_diag(b)
            e["mass_drift_mixed"] = abs(da["mass"] / m0a - 1.0)
            e["mass_drift_fp64"] = abs(db["mass"] / m0b - 1.0)
            e["nonfinite_mixed"] = da["nonfinite"]
            report[n] = e
    finally:
        thor.thor_state_destroy(a)
        thor.thor_state_destroy(b)
        thor.thor_grid_destroy(grid)
    out = report_dir()
    if out:
        json.dump(report, open(os.path.join(out, "mixed_long.json"), "w"), indent=1)
    print(report)
    r10, r100, r1000 = report[10], report[100], report[1000]
    assert r10["rho_rel_l2"] < 1e-6 and r10["T_rel_l2"] < 1e-6 and r10["vh_max_abs"] < 2e-3, r10
    assert r100["rho_rel_l2"] < 1e-5 and r100["T_rel_l2"] < 1e-5 and r100["vh_max_abs"] < 0.05, r100
    assert r1000["nonfinite_mixed"] == 0
    assert r1000["mass_drift_mixed"] < 1e-6 and r1000["mass_drift_fp64"] < 1e-12, r1000


@pytest.mark.parametrize("precision", [thor.THOR_FP64, thor.THOR_MIXED])
@pytest.mark.parametrize("device_buffer", [False, True])
def test_restart_from_checkpoint_is_bit_exact(precision, device_buffer):
    """Stepping 3 + 3 large steps through a raw checkpoint (saved to host or
    device memory, loaded into a fresh state) equals 6 uninterrupted steps
    bit for bit; a checkpoint does not load into a state of another size."""
    wl = wls.HS_G4
    grid = _grid(wl)
    mk = lambda: thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, precision), None)
    a, b = mk(), mk()
    c = None
    try:
        thor.thor_step(a, 6, wl.n_small, wl.dt)
        thor.thor_step(b, 3, wl.n_small, wl.dt)
        n = thor.thor_checkpoint_bytes(b)
        buf = torch.empty(n, dtype=torch.uint8, device="cuda") if device_buffer else None
        buf = thor.thor_checkpoint_save(b, buf)
        c = mk()
        thor.thor_checkpoint_load(c, buf)
        thor.thor_step(c, 3, wl.n_small, wl.dt)
        for f in FIELDS:
            assert np.array_equal(thor.thor_state_get(a, f, wl.ncol, wl.nv),
                                  thor.thor_state_get(c, f, wl.ncol, wl.nv)), f
        with pytest.raises(thor.ThorError):
            thor.thor_checkpoint_load(c, buf[:-1])
        # the stored deviations are relative to the saving state's reference
        # column: a state of the same size with another start temperature or
        # planet refuses the checkpoint and keeps its fields
        for other in (wl.with_(T0=wl.T0 + 10.0), wl.with_(planet=wls.EARTH_TABLE1)):
            d = thor.thor_state_init(grid, planet_struct(other.planet), init_struct(other, precision), None)
            try:
                before = thor.thor_state_get(d, thor.THOR_FIELD_RHO, wl.ncol, wl.nv)
                with pytest.raises(thor.ThorError) as e:
                    thor.thor_checkpoint_load(d, buf)
                assert e.value.status == thor.THOR_EINVAL
                assert np.array_equal(before, thor.thor_state_get(d, thor.THOR_FIELD_RHO, wl.ncol, wl.nv))
            finally:
                thor.thor_state_destroy(d)
    finally:
        for s_ in (a, b, c):
            if s_ is not None:
                thor.thor_state_destroy(s_)
        thor.thor_grid_destroy(grid)


@pytest.mark.parametrize("precision, compensated", [(thor.THOR_FP64, 0), (thor.THOR_MIXED, 1),
                                                     (thor.THOR_MIXED, 0)])
def test_restart_through_float64_fields(precision, compensated):
    """The same restart through thor_state_get / thor_state_set: bit for bit
    for a plain float state (a float32 deviation plus the float64 reference
    is exact in float64). In float64 storage, and in a compensated float
    state (a pair of about 48 bits), reference + deviation rounds to the
    last place of the full value (rho theta near 300, p near 1e5); three
    large steps carry that into the small momentum field at about 4e-13 of
    its largest value, so the bound there is 1e-11."""
    wl = wls.HS_G4
    grid = _grid(wl)

    def mk():
        st = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, precision), None)
        if precision == thor.THOR_MIXED:
            thor.thor_tune(st, thor.THOR_TUNE_COMPENSATED, compensated)
        return st
    a, b = mk(), mk()
    c = None
    try:
        thor.thor_step(a, 6, wl.n_small, wl.dt)
        thor.thor_step(b, 3, wl.n_small, wl.dt)
        saved = [thor.thor_state_get(b, f, wl.ncol, wl.nv) for f in FIELDS]
        c = mk()
        for f, x in zip(FIELDS, saved):
            thor.thor_state_set(c, f, x)
        thor.thor_step(c, 3, wl.n_small, wl.dt)
        for f in FIELDS:
            x = thor.thor_state_get(a, f, wl.ncol, wl.nv)
            y = thor.thor_state_get(c, f, wl.ncol, wl.nv)
            if precision == thor.THOR_MIXED and not compensated:
                assert np.array_equal(x, y), f
            else:
                assert np.max(np.abs(x - y)) <= 1e-11 * np.max(np.abs(x)), f
    finally:
        for s_ in (a, b, c):
            if s_ is not None:
                thor.thor_state_destroy(s_)
        thor.thor_grid_destroy(grid)


def test_bounded_device_wait_gives_up_and_the_context_stays_usable():
    """A device wait on a barrier that nothing completes runs out after its
    limit and reports it; with the arrival it completes at once; afterwards
    the same context steps a state normally."""
    import time
    t0 = time.perf_counter()
    assert thor.thor_wait_selftest(0, 20000) == 1
    assert time.perf_counter() - t0 >= 0.015
    assert thor.thor_wait_selftest(1, 20000) == 0
    wl = wls.HS_G4
    grid = _grid(wl)
    st = thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl, thor.THOR_MIXED), None)
    try:
        thor.thor_step(st, 1, wl.n_small, wl.dt)
        assert thor.thor_diag(st)["nonfinite"] == 0
    finally:
        thor.thor_state_destroy(st)
        thor.thor_grid_destroy(grid)

