"""Test harness: runs one workload on the CUDA library (through the C ABI)
and on the oracle, with a column permutation between their numberings found
by matching grid coordinates. Test infrastructure only."""

import numpy as np
from scipy.spatial import cKDTree

import paper_1607_05535_gb300 as thor
from conftest import oracle_grid
from oracle import dycore as dc
from oracle import operators as op
import workloads as wls

FORCING = {"none": thor.THOR_FORCING_NONE, "held_suarez": thor.THOR_FORCING_HELD_SUAREZ,
           "hot_jupiter": thor.THOR_FORCING_HOT_JUPITER}


def planet_struct(P):
    return thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)


def init_struct(wl, precision=thor.THOR_FP64, hyper=1, divdamp=1, shallow=0, hydrostatic=0, profile=0, vorder=1,
                anelastic=0):
    return thor.thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, FORCING[wl.forcing], wl.hj_dT,
                          precision, hyper, divdamp, shallow, hydrostatic, profile, vorder, anelastic)


class Pair:
    """A workload on both sides. ``perm[c]`` is the oracle index of library
    column c."""

    def __init__(self, wl, precision=thor.THOR_FP64, hyper=True, divdamp=True, stream=None, shallow=False,
                 hydrostatic=False, profile=False, vorder=1, anelastic=False):
        self.wl = wl
        sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, wl.spring_tol, wl.spring_max_iter)
        self.grid = thor.thor_grid_create(wl.glevel, wl.nv, wl.planet.radius, wl.z_top, sp)
        self.state = thor.thor_state_init(self.grid, planet_struct(wl.planet),
                                          init_struct(wl, precision, int(hyper), int(divdamp), int(shallow),
                                                      int(hydrostatic),
                                                      thor.THOR_PROFILE_HELD_SUAREZ if profile else 0, vorder,
                                                      int(anelastic)),
                                          stream)
        self.ncol, self.nv = wl.ncol, wl.nv
        self.profile = "held_suarez" if profile else None
        P = wl.planet
        G = oracle_grid(wl.glevel, max_iter=wl.spring_max_iter, tol=wl.spring_tol)
        pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
        self.model = dc.Model(G, op.VerticalGrid(wl.nv, wl.z_top, P.radius, shallow=shallow), pl, forcing=wl.forcing,
                              hj_dT=wl.hj_dT, hyperdiffusion=hyper, divergence_damping=divdamp,
                              hydrostatic=hydrostatic, vorder=vorder, anelastic=anelastic)
        d, self.perm = cKDTree(G.points).query(thor.thor_grid_points(self.grid))
        assert d.max() < 1e-11 and len(np.unique(self.perm)) == self.ncol

    def close(self):
        thor.thor_state_destroy(self.state)
        thor.thor_grid_destroy(self.grid)

    def oracle_initial(self):
        u = None
        if self.wl.noise_amp > 0:
            u = np.empty((self.ncol, self.nv))
            u[self.perm] = wls.temperature_noise(self.wl)
        return dc.initial_state(self.model, self.wl.T0, self.wl.p_surf, self.wl.noise_amp, u, profile=self.profile)

    def get(self):
        """Library state as an oracle State in oracle column order."""
        g = lambda f: thor.thor_state_get(self.state, f, self.ncol, self.nv)
        out = dc.State(np.empty((self.ncol, self.nv)), np.empty((self.ncol, self.nv, 3)),
                       np.empty((self.ncol, self.nv + 1)), np.empty((self.ncol, self.nv)))
        out.rho[self.perm] = g(thor.THOR_FIELD_RHO)
        out.M[self.perm] = g(thor.THOR_FIELD_MOM)
        out.W[self.perm] = g(thor.THOR_FIELD_W)
        out.Th[self.perm] = g(thor.THOR_FIELD_RHOTHETA)
        return out

    def set(self, X):
        thor.thor_state_set(self.state, thor.THOR_FIELD_RHO, X.rho[self.perm])
        thor.thor_state_set(self.state, thor.THOR_FIELD_MOM, X.M[self.perm])
        thor.thor_state_set(self.state, thor.THOR_FIELD_W, X.W[self.perm])
        thor.thor_state_set(self.state, thor.THOR_FIELD_RHOTHETA, X.Th[self.perm])


def rel_l2(a, b, floor=0.0):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor))


def field_errors(A, B):
    """Relative L2 per field of A against B (oracle) and max-abs on W."""
    return dict(rho=rel_l2(A.rho, B.rho), M=rel_l2(A.M, B.M, 1e-300), W=rel_l2(A.W, B.W, 1e-300),
                Th=rel_l2(A.Th, B.Th), W_maxabs=float(np.max(np.abs(A.W - B.W))))


def change_errors(A, B, X0):
    """Per element, per field: max |A - B| over the largest change of the
    oracle's field from its start, max |B - X0|. A localised error (a
    pentagon, a rhombus edge) cannot hide in this the way it can in a
    relative L2 dominated by the hydrostatic background of rho and rho theta."""
    out = {}
    for f in ("rho", "M", "W", "Th"):
        a, b, x0 = getattr(A, f), getattr(B, f), getattr(X0, f)
        change = float(np.max(np.abs(b - x0)))
        err = float(np.max(np.abs(a - b)))
        out[f] = err / change if change > 0 else err
    return out


def moving_start(pair, X, seed=11, amp=5.0):
    """X (an oracle state at rest) with a smooth motion added and injected into
    both sides: horizontal momentum rho (u0 z x r + a random projected
    field of 1% of it) with u0 = amp m/s at the equator, vertical momentum of
    1e-3 kg m^-2 s^-1 on the interior interfaces. From rest with density-only
    noise the pressure is horizontally uniform and the first small step
    leaves M at zero, where the oracle keeps float64 rounding noise."""
    from oracle import operators as op
    rng = np.random.default_rng(seed)
    r = pair.model.rhat
    rot = np.cross(np.array([0.0, 0.0, 1.0])[None, :], r)
    v = amp * rot[:, None, :] + 0.01 * amp * op.project_h(r, rng.standard_normal(X.M.shape))
    X.M[:] = X.rho[..., None] * v
    X.W[:, 1:-1] = 1e-3 * rng.standard_normal((X.W.shape[0], X.W.shape[1] - 2))
    pair.set(X)
    return X

