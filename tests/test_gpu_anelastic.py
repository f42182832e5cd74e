"""The anelastic switch on the GPU path (thor_init.anelastic, Sec. 3;
readings A-1..A-6 of oracle/anelastic.py) against the oracle.

The library solves the pressure equation iteratively (float64 BiCGStab to a
true relative residual of 1e-13), the oracle directly (sparse LU with
iterative refinement). The operator's condition number (about 1e7 at glevel
3 x 12 levels: the vertical coupling exceeds the horizontal by (dx/dz)^2)
turns the two solvers' float64 residuals into p' differences in its
near-null, horizontally smooth modes, which reach the momentum at about 1e-8
(measured 7.6e-9 relative L2 on M, 1.4e-11 on W, 1.2e-14 on rho theta after
two large steps); the float64 gates are 3e-8 on M, 1e-9 on W and 1e-12 on
rho theta.
The mixed path stays within the mixed-mode gates; the divergence of an
unforced float64 state is checked with the oracle's operators."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from harness import Pair, field_errors, init_struct, planet_struct
from oracle import anelastic as an
from oracle import dycore as dc
import workloads as wls

WL = wls.HS_G4.with_(name="hs_g3_L12", glevel=3, nv=12, n_large=2, noise_amp=0.5, dt=900.0)


class AnelasticPair(Pair):
    """A Pair whose both sides run the anelastic switch from the same start:
    rho the reference column and the seeded temperature noise dT as
    theta' = theta0 dT / T0."""

    def __init__(self, wl, precision):
        super().__init__(wl, precision=precision, anelastic=True)

    def oracle_initial(self):
        u = np.empty((self.ncol, self.nv))
        u[self.perm] = wls.temperature_noise(self.wl)
        rho0, theta0 = an.reference_column(self.model, self.wl.T0, self.wl.p_surf)
        dT = self.wl.noise_amp * (2.0 * u - 1.0)
        return an.anelastic_start(self.model, self.wl.T0, self.wl.p_surf, theta_prime=theta0[None, :] * dT / self.wl.T0)


def test_float64_matches_oracle():
    p = AnelasticPair(WL, thor.THOR_FP64)
    try:
        X = p.oracle_initial()
        start = p.get()
        assert field_errors(start, X)["rho"] < 1e-14 and field_errors(start, X)["Th"] < 1e-14
        ref = dc.run(p.model, X, 2, WL.n_small, WL.dt)
        thor.thor_step(p.state, 2, WL.n_small, WL.dt)
        got = p.get()
        e = field_errors(got, ref)
        assert np.abs(ref.M).max() > 1e-3                      # the buoyancy moved the air
        assert e["rho"] < 1e-14, e
        assert e["M"] < 3e-8 and e["W"] < 1e-9 and e["Th"] < 1e-12, e
    finally:
        p.close()


def test_float64_state_is_divergence_free():
    """Without forcing (the Held-Suarez friction acts on the momentum after
    the last projection of a step, so a forced state carries the friction's
    divergence in the boundary layer) the GPU state after two large steps
    satisfies the discrete constraint div(rho0 v) = 0 of the oracle's
    operators to 1e-9 of a horizontal divergence term."""
    p = AnelasticPair(WL.with_(forcing="none"), thor.THOR_FP64)
    try:
        p.oracle_initial()
        thor.thor_step(p.state, 2, WL.n_small, WL.dt)
        got = p.get()
        assert np.abs(got.M).max() > 1e-3
        D = an.divergence(p.model, got.M, got.W)
        scale = np.abs(got.M).max() / p.model.vg.rc[0] * 1e3    # a horizontal divergence term's size
        assert np.abs(D).max() < 1e-9 * scale, (np.abs(D).max(), scale)
    finally:
        p.close()


def test_mixed_within_gates():
    p = AnelasticPair(WL, thor.THOR_MIXED)
    try:
        X = p.oracle_initial()
        ref = dc.run(p.model, X, 2, WL.n_small, WL.dt)
        thor.thor_step(p.state, 2, WL.n_small, WL.dt)
        A = p.get()
        rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel(A.Th, ref.Th) < 1e-6
        assert np.abs(A.M / A.rho[..., None] - ref.M / ref.rho[..., None]).max() < 2e-3
    finally:
        p.close()


def test_refused_combinations():
    P = WL.planet
    grid = thor.thor_grid_create(2, 8, P.radius, 2.0e4, thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, 10))
    try:
        bad = init_struct(WL, thor.THOR_FP64, hydrostatic=1)
        bad.anelastic = 1
        with pytest.raises(thor.ThorError):
            thor.thor_state_init(grid, planet_struct(P), bad, None)
        ok = init_struct(WL, thor.THOR_MIXED)
        ok.anelastic = 1
        s = thor.thor_state_init(grid, planet_struct(P), ok, None)
        try:
            with pytest.raises(thor.ThorError):
                thor.thor_tune(s, thor.THOR_TUNE_COMPENSATED, 1)
            ens = thor.thor_ensemble_create([s], None)
            try:
                with pytest.raises(thor.ThorError):
                    thor.thor_ensemble_step(ens, 1, [6], [900.0])
            finally:
                thor.thor_ensemble_destroy(ens)
        finally:
            thor.thor_state_destroy(s)
    finally:
        thor.thor_grid_destroy(grid)
