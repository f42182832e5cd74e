"""Edge cases of the CUDA path against the oracle: the smallest grids
(glevel 0: the 12 icosahedron vertices, all pentagons, fewer columns than a
warp; glevel 1: 42 columns), the fewest levels (nv = 2: one interior
interface, so one sweep of the column solve is empty and the junction is a
single row), odd level counts (the two sweeps of unequal length), and the
largest column the kernels accept (nv = 128, THOR_MAX_NV: the staged solve's
planes fill 165 KB of shared memory). One Held-Suarez large step from the
seeded noisy start, float64 to 1e-10 relative per field; the mixed mode
(TMA-staged solve) within the absolute gates of the mixed tests; nv = 129 is
refused. The cases run in turn, so a state with fewer levels follows one with
128 and must leave the shared-memory limit of the column kernels raised."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from harness import Pair, field_errors, init_struct, planet_struct
from oracle import dycore as dc
import workloads as wls

CASES = [(1, 128), (0, 2), (0, 5), (1, 3), (1, 7), (2, 2)]   # 128 levels first: the others follow it


def _wl(glevel, nv):
    """At most 2 km per layer: with thicker layers the discretely balanced
    isothermal column of the start (each interface's pressure from the one
    below by a two-point balance) turns negative, g dz / (R_d T) > 2."""
    return wls.HS_G4.with_(name="edge_g%d_L%d" % (glevel, nv), glevel=glevel, nv=nv, n_large=1,
                           z_top=min(36.0e3, 2.0e3 * nv))


@pytest.mark.parametrize("glevel,nv", CASES)
def test_edge_parity_fp64(glevel, nv):
    wl = _wl(glevel, nv)
    p = Pair(wl)
    try:
        X = p.oracle_initial()
        ref = dc.run(p.model, X, 1, wl.n_small, wl.dt)
        thor.thor_step(p.state, 1, wl.n_small, wl.dt)
        e = field_errors(p.get(), ref)
        assert e["rho"] < 1e-10 and e["Th"] < 1e-10 and e["M"] < 1e-10, e
        # W, small after one step, is the difference of the nearly equal vertical
        # terms of size g rho dtau, which float64 rounds at about 1e-16 of that
        w_scale = wl.planet.gravity * float(np.abs(ref.rho).max()) * wl.dt / wl.n_small
        assert e["W"] < 1e-10 or e["W_maxabs"] < 1e-12 * w_scale, e
    finally:
        p.close()


@pytest.mark.parametrize("glevel,nv", CASES)
def test_edge_mixed(glevel, nv):
    from test_gpu_mixed import GATES, field_report
    wl = _wl(glevel, nv)
    p = Pair(wl, precision=thor.THOR_MIXED)
    try:
        ref = dc.run(p.model, p.oracle_initial(), 1, wl.n_small, wl.dt)
        thor.thor_step(p.state, 1, wl.n_small, wl.dt)
        rep = field_report(p, p.get(), ref)
        for k, g in GATES.items():
            if k != "vh_rel":      # relative to winds of 1e-3 m/s after one step from rest
                assert rep[k] < g, (k, rep)
    finally:
        p.close()


def test_too_many_levels_refused():
    wl = _wl(1, 129)
    grid = thor.thor_grid_create(1, 129, wl.planet.radius, wl.z_top, thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, 5))
    try:
        with pytest.raises(thor.ThorError) as e:
            thor.thor_state_init(grid, planet_struct(wl.planet), init_struct(wl))
        assert e.value.status == thor.THOR_EINVAL
    finally:
        thor.thor_grid_destroy(grid)
