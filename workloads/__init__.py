"""Seeded synthetic workloads: parameter sets and input random numbers.

This module holds only inputs (planet constants, grid and run sizes, seeds)
and one counter-based random generator. It holds none of the method's
arithmetic. Both the CUDA path's tests and bench and the oracle draw their
inputs from here; the CUDA library implements the same generator itself from
its published definition (SplitMix64, Steele, Lea and Flood 2014).

Planet constants: Table 1 of the paper, with the benchmark configurations'
own values where they differ (Earth cp = 1005, Rd = 287; hot-Jupiter g = 9.42).
"""

from dataclasses import dataclass, replace

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output for the state ``x`` (uint64 numpy array): the state is
    advanced by the golden-ratio increment, then mixed."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(seed, counter):
    """u in [0, 1) from the top 53 bits of splitmix64(seed XOR counter)."""
    s = np.uint64(seed & MASK64)
    z = splitmix64(np.asarray(counter, dtype=np.uint64) ^ s)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class PlanetParams:
    radius: float
    omega: float
    gravity: float
    Rd: float
    cp: float
    p_ref: float = 1.0e5
    dt_paper: float = 1000.0     # the paper's time step for this planet (Sec. 6)
    tau_d: float = 6.46e3        # Table 1 diffusion time scale

    @property
    def diff_D(self):
        """Nondimensional diffusion parameter from Eqs. kd, tau_d."""
        return self.dt_paper / (32.0 * self.tau_d)


EARTH = PlanetParams(radius=6.371e6, omega=7.292e-5, gravity=9.8, Rd=287.0, cp=1005.0,
                     dt_paper=1000.0, tau_d=6.46e3)
HOT_JUPITER = PlanetParams(radius=1.0e8, omega=2.1e-5, gravity=9.42, Rd=3779.0, cp=13226.0,
                           dt_paper=600.0, tau_d=941.2)
# Table 1 of the paper as printed (the long runs of Sec. 6 use these)
EARTH_TABLE1 = PlanetParams(radius=6.371e6, omega=7.292e-5, gravity=9.8, Rd=287.04, cp=1004.6,
                            dt_paper=1000.0, tau_d=6.46e3)
HOT_JUPITER_TABLE1 = PlanetParams(radius=1.0e8, omega=2.1e-5, gravity=8.0, Rd=3779.0, cp=13226.5,
                                  dt_paper=600.0, tau_d=941.2)


@dataclass(frozen=True)
class Workload:
    name: str
    glevel: int
    nv: int
    z_top: float
    planet: PlanetParams
    T0: float
    p_surf: float
    noise_amp: float
    seed: int
    forcing: str              # "none" | "held_suarez" | "hot_jupiter"
    dt: float
    n_small: int
    n_large: int
    spring_max_iter: int = 10
    spring_tol: float = 0.0
    hj_dT: float = 300.0

    @property
    def ncol(self):
        return 10 * 4 ** self.glevel + 2

    @property
    def cells(self):
        return self.ncol * self.nv

    @property
    def substeps_per_large(self):
        return 1 + self.n_small // 2 + self.n_small

    def with_(self, **kw):
        return replace(self, **kw)


# Held-Suarez Earth, glevel 4 x 20 levels, 36 km top, 300 K at rest with
# +-0.1 K seeded noise, dt 1800 s, 6 small steps, 10 large steps.
HS_G4 = Workload("held_suarez_g4_L20", glevel=4, nv=20, z_top=36.0e3, planet=EARTH, T0=300.0,
                 p_surf=1.0e5, noise_amp=0.1, seed=1234, forcing="held_suarez", dt=1800.0,
                 n_small=6, n_large=10, spring_max_iter=10)

# Held-Suarez Earth, glevel 6 (40962 columns) x 32 levels, dt 600 s,
# 8 small steps (13 small steps per large step).
HS_G6 = Workload("held_suarez_g6_L32", glevel=6, nv=32, z_top=36.0e3, planet=EARTH, T0=300.0,
                 p_surf=1.0e5, noise_amp=0.1, seed=1234, forcing="held_suarez", dt=600.0,
                 n_small=8, n_large=1000, spring_max_iter=10)


def hot_jupiter_contrast(seed=0xC0FFEE):
    """Day-night equilibrium contrast drawn from U[500, 1000] K."""
    return 500.0 + 500.0 * float(uniform01(seed, 0))


def hot_jupiter_top(planet=HOT_JUPITER, T=1600.0, p_bottom=220.0e5, p_top=1.0e2):
    """Altitude where an isothermal atmosphere falls from p_bottom to p_top."""
    return planet.Rd * T / planet.gravity * np.log(p_bottom / p_top)


HJ_G6 = Workload("hot_jupiter_g6_L32", glevel=6, nv=32, z_top=float(hot_jupiter_top()),
                 planet=HOT_JUPITER, T0=1600.0, p_surf=220.0e5, noise_amp=0.0, seed=0xC0FFEE,
                 forcing="hot_jupiter", dt=300.0, n_small=6, n_large=1000, spring_max_iter=10,
                 hj_dT=hot_jupiter_contrast())


def temperature_noise(wl, ncol=None):
    """u (ncol, nv) for the initial temperature noise, indexed by the canonical
    (rhombus-major) column order of the CUDA library: counter = col * nv + k."""
    ncol = wl.ncol if ncol is None else ncol
    idx = np.arange(ncol, dtype=np.uint64)[:, None] * np.uint64(wl.nv) + np.arange(wl.nv, dtype=np.uint64)[None, :]
    return uniform01(wl.seed, idx)


# Batched ensemble: 64 independent Held-Suarez atmospheres x 32 levels on
# glevels drawn from {3, 4, 5}, radius and rotation rate each drawn
# log-uniform over [0.1, 10] x Earth from one seed. The time step keeps the
# Courant numbers of the glevel-5 Earth case (dt 1200 s, 8 small steps): it
# scales with the grid spacing, radius * 2^-glevel, and is capped at
# 1 / (4 Omega) so that the explicit Coriolis term stays well inside the RK3
# stability region.
ENSEMBLE_SEED = 42


@dataclass(frozen=True)
class EnsembleMember:
    glevel: int
    planet: PlanetParams
    dt: float
    n_small: int = 8

    @property
    def ncol(self):
        return 10 * 4 ** self.glevel + 2


def ensemble_members(n=64, seed=ENSEMBLE_SEED, glevels=(3, 4, 5), n_small=8):
    out = []
    for i in range(n):
        u = [float(uniform01(seed, 3 * i + j)) for j in range(3)]
        g = glevels[min(int(u[0] * len(glevels)), len(glevels) - 1)]
        radius = EARTH.radius * 10.0 ** (2.0 * u[1] - 1.0)
        omega = EARTH.omega * 10.0 ** (2.0 * u[2] - 1.0)
        dt = min(1200.0 * (radius / EARTH.radius) * 2.0 ** (5 - g), 0.25 / omega)
        out.append(EnsembleMember(g, replace(EARTH, radius=radius, omega=omega), dt, n_small))
    return out


ENSEMBLE_NV, ENSEMBLE_Z_TOP = 32, 36.0e3
