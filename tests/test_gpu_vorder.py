"""Higher-order vertical interpolation on the GPU path (thor_init.vorder,
Sec. 2.1 with k = 2 and 3 in the explicit terms, reading L-2) against the
float64 oracle with the same order: every field within 1e-10 relative L2
and every element within 1e-8 of its field's largest change, from a moving
start, two large steps; with the shallow-atmosphere switch as well; the
mixed path within the mixed-mode gates; sizes the order cannot serve are
refused."""

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

WL = wls.HS_G4.with_(name="hs_g3_L12", glevel=3, nv=12, n_large=2)


@pytest.mark.parametrize("vorder, shallow", [(2, False), (3, False), (3, True)])
def test_float64_matches_oracle(vorder, shallow):
    p = Pair(WL, vorder=vorder, shallow=shallow)
    try:
        X = moving_start(p, p.oracle_initial())
        ref = dc.run(p.model, X, 2, WL.n_small, WL.dt)
        thor.thor_step(p.state, 2, WL.n_small, WL.dt)
        got = p.get()
        e = field_errors(got, ref)
        assert max(e["rho"], e["Th"], e["M"], e["W"]) < 1e-10, e
        c = change_errors(got, ref, X)
        assert max(c.values()) < 1e-8, c
        # the order matters: the linear model moves elsewhere by far more
        lin = dc.Model(p.model.grid, p.model.vg, p.model.planet, forcing=WL.forcing, vorder=1)
        ref1 = dc.run(lin, X, 2, WL.n_small, WL.dt)
        assert field_errors(ref1, ref)["M"] > 1e3 * max(e["M"], 1e-16)
    finally:
        p.close()


def test_mixed_within_gates():
    p = Pair(WL, precision=thor.THOR_MIXED, vorder=3)
    try:
        X = moving_start(p, p.oracle_initial())
        ref = dc.run(p.model, X, 2, WL.n_small, WL.dt)
        thor.thor_step(p.state, 2, WL.n_small, WL.dt)
        A = p.get()
        rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel(A.rho, ref.rho) < 1e-6 and rel(A.Th, ref.Th) < 1e-6
        assert np.abs(A.M / A.rho[..., None] - ref.M / ref.rho[..., None]).max() < 2e-3
    finally:
        p.close()


def test_order_needs_enough_levels():
    P = WL.planet
    grid = thor.thor_grid_create(2, 3, P.radius, 10.0e3, thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, 10))
    try:
        for bad in (3, 4, -1):
            with pytest.raises(thor.ThorError):
                thor.thor_state_init(grid, planet_struct(P), init_struct(WL, vorder=bad), None)
        s = thor.thor_state_init(grid, planet_struct(P), init_struct(WL, vorder=2), None)
        thor.thor_state_destroy(s)
    finally:
        thor.thor_grid_destroy(grid)
