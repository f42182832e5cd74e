"""Oracle dynamical core (Sec. 3-4), float64, numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Prognostic state (Arakawa-A in the horizontal, Sec. 2.2; vertical momentum at
the layer interfaces, Sec. 3):

  rho  (N, nv)      density at the centres
  M    (N, nv, 3)   horizontal momentum rho v_h as a Cartesian vector
  W    (N, nv+1)    vertical momentum rho v_r at the interfaces, W = 0 at the
                    bottom and top (rigid lid, Sec. 3)
  Th   (N, nv)      rho theta

Readings:

R1  Time stepping. Sec. 3 calls each of the three Wicker-Skamarock stages a
    "large time step" when it gives the small-step counts (1 step of dt/3,
    n/2 steps of dt/n, n steps of dt/n). We read the small-step equations
    (Eqs. dens2, mom2, momr2, pt2) the same way: Phi^[t] there is the state
    of the current stage Phi^(s), the slow terms and the linearisation
    coefficients are evaluated at Phi^(s), and the deviations
    Phi* = Phi - Phi^(s) start each stage at Phi^t - Phi^(s), so the inner
    loop always integrates from Phi^t and the stage ends at
    Phi^(s+1) = Phi^(s) + Phi*. With the acoustic terms frozen this is exactly
    the RK3 update Phi^(s+1) = Phi^t + dt_s R(Phi^(s)).
R2  Eq. pt2: (rho v)^[tau+dtau] is the total momentum Phi^(s) + Phi*, and the
    radial operator is the deep one, r^-2 d(r^2 .)/dr, as in Eq. dens2.
R3  Eq. vr22 is garbled. The vertical system is instead the exact discrete
    substitution of the discrete Eqs. dens2 and pt2 into the discrete
    Eq. momr2, with p* advanced linearly, p*+ = p* + Pi (Th+ - Th),
    Pi = (cp/cv) p^(s)/Th^(s). Unknown: W* at the interior interfaces.
    After the solve rho* and Th follow exactly from Eqs. dens2 and pt2 and
    p* from the nonlinear Eq. theta_to_p.
R4  Hyperdiffusion (Sec. 4, Eqs. diff_rho ... diff_p): every momentum
    component is rho-weighted, F_M = -lap(rho K_d lap v_h) component-wise and
    projected, like Eq. diff_vr; the third line of Eq. diff_vz is F_vhz. F_p
    enters as a slow tendency of rho theta, F_Th = Th/(gamma p) F_p.
R5  The divergence damping of Eqs. diff_vx-vz, printed -K_d lap(grad_h D)
    with D the 3-D divergence of the momentum, is evaluated every small step
    (Sec. 4) from the current total momentum, in the order -K_d grad_h(lap D):
    on the sphere the projected Cartesian Laplacian of a gradient field is
    the gradient of the Laplacian (Weitzenboeck identity, Ricci curvature 1),
    so both orders have one continuum limit; the discrete gradient of the
    Sec. 4 Laplacian is the more accurate (11% against 13% relative L2 at
    glevel 3, 9.5% against 12% at glevel 4, on a closed-form field) and needs
    one scalar instead of a vector per cell between the two stencils.
R6  Advection and Coriolis (Sec. 3): A_j = div(rho v v_j) for the three
    Cartesian components of the full velocity v = M/rho + (W/rho) r, then
    projected by Eqs. proj_h / proj_r; their radial parts are interpolated
    to the interfaces.
R7  K_d = D dbar^4 / dt (Eq. kd) with dbar from Eq. grid_qts; the
    nondimensional D of a planet follows from its Table 1 diffusion time
    scale through Eq. tau_d at the paper's own time step.
L-2 Higher-order vertical interpolation (Sec. 2.1 implements the Lagrange
    polynomial of any order k and runs k = 1): with vorder = k > 1 the
    explicit terms interpolate with order k (reading L-1 for the nodes): the
    velocity at the interfaces for the vertical advection, W at the centres
    for the full momentum (advection, Coriolis), the radial advection and
    Coriolis at the interfaces, and rho at the interfaces of the vertical
    hyperdiffusion. The terms that enter the implicit vertical system keep
    k = 1: rho at the interfaces in the gravity term, theta at the
    interfaces, and the pressure gradient, so the vertical system stays
    tridiagonal, the discrete hydrostatic balance of a resting column holds
    exactly and a uniform theta stays uniform.
H1  Hydrostatic switch (Sec. 3 lists the hydrostatic approximation among
    those the model implements but does not use: the vertical pressure
    gradient balances gravity). Read as a factor delta on the vertical
    momentum's inertia: delta = 0 drops dW/dt with the vertical advection,
    the radial Coriolis part and the diffusion of W, so that Eq. momr2
    becomes 0 = -dp/dr - g rho at the new small-step state. The vertical
    system of R3 keeps its form with the identity term and W* on the
    right-hand side scaled by delta: W is diagnosed every small step so that
    the new state is in discrete hydrostatic balance (linearised p*, as R3).
"""

from dataclasses import dataclass, field

import numpy as np

from . import operators as op
from .grid import mean_resolution


@dataclass
class Planet:
    radius: float
    omega: float
    gravity: float
    Rd: float
    cp: float
    p_ref: float = 1.0e5          # Sec. 3: p_ref = 1 bar
    diff_D: float = 0.0           # nondimensional diffusion parameter of Eq. kd

    @property
    def cv(self):
        return self.cp - self.Rd

    @property
    def gamma(self):
        return self.cp / self.cv

    @property
    def kappa(self):
        return self.Rd / self.cp


def diffusion_parameter(dt_paper, tau_d):
    """Eqs. kd and tau_d: tau_d = dbar^4/(32 K_d) and K_d = D dbar^4/dt give
    D = dt / (32 tau_d)."""
    return dt_paper / (32.0 * tau_d)


@dataclass
class State:
    rho: np.ndarray
    M: np.ndarray
    W: np.ndarray
    Th: np.ndarray

    def copy(self):
        return State(self.rho.copy(), self.M.copy(), self.W.copy(), self.Th.copy())


@dataclass
class Model:
    grid: object
    vg: object
    planet: Planet
    forcing: str = "none"          # "none" | "held_suarez" | "hot_jupiter"
    hj_dT: float = 300.0           # Eq. teq-hj day-night contrast
    hyperdiffusion: bool = True
    divergence_damping: bool = True
    hydrostatic: bool = False      # reading H1
    vorder: int = 1                # reading L-2: order k of the explicit vertical interpolations
    anelastic: bool = False        # readings A-1..A-6 (oracle.anelastic)
    reference: tuple = None        # (rho0, theta0) of the anelastic reference column, (nv,) each
    Kd_fixed: float = None         # a fixed K_d instead of Eq. kd (tests)
    rhat: np.ndarray = field(init=False)

    def __post_init__(self):
        self.rhat = self.grid.points

    def Kd(self, dt):
        """Eq. kd."""
        if self.Kd_fixed is not None:
            return self.Kd_fixed
        _, dbar, _ = mean_resolution(self.grid.glevel, self.planet.radius)
        return self.planet.diff_D * dbar ** 4 / dt


# ------------------------------------------------------------ thermodynamics

def pressure(planet, Th):
    """Eq. pressure: p = p_ref (Rd rho theta / p_ref)^(cp/cv)."""
    return planet.p_ref * (planet.Rd * Th / planet.p_ref) ** planet.gamma


def rhotheta_from_p(planet, p):
    """Inverse of Eq. pressure."""
    return planet.p_ref / planet.Rd * (p / planet.p_ref) ** (1.0 / planet.gamma)


def temperature(planet, rho, p):
    """Ideal gas, Sec. 3: p = rho Rd T."""
    return p / (rho * planet.Rd)


# ------------------------------------------------------------- slow terms

def hyperdiffusion(model, X, p, Kd):
    """Sec. 4, Eqs. diff_rho ... diff_p with readings R4, R7."""
    g, vg, pl = model.grid, model.vg, model.planet
    rho_i = op.interp_to_interfaces(vg, X.rho, model.vorder)
    vh = X.M / X.rho[..., None]
    vr = np.zeros_like(X.W)
    vr[:, 1:-1] = X.W[:, 1:-1] / rho_i[:, 1:-1]
    T = temperature(pl, X.rho, p)

    F_rho = -op.lap_levels(g, vg, Kd * op.lap_levels(g, vg, X.rho))
    lv = op.vlap_levels(g, vg, vh)
    F_M = -op.vlap_levels(g, vg, X.rho[..., None] * Kd * lv)
    F_M = op.project_h(model.rhat, F_M)
    F_W = np.zeros_like(X.W)
    inner = op.lap_levels(g, vg, vr, at_interfaces=True)
    F_W[:, 1:-1] = -op.lap_levels(g, vg, rho_i * Kd * inner, at_interfaces=True)[:, 1:-1]
    F_p = -pl.Rd * op.lap_levels(g, vg, X.rho * Kd * op.lap_levels(g, vg, T))
    F_Th = X.Th / (pl.gamma * p) * F_p
    return F_rho, F_M, F_W, F_Th


def _shallow_advection_coriolis(model, X, Wc):
    """Advection and Coriolis under the shallow-atmosphere approximation of
    Sec. 3 with the "traditional approximation" it names: reading S-2, only
    the local vertical component of Omega acts, on the horizontal momentum,
    C_h = 2 Omega (z . r) r x M_h, and nothing on the vertical momentum;
    reading S-3, the metric terms that the traditional approximation drops
    for angular-momentum conservation (u w / r, v w / r in the horizontal,
    (u^2 + v^2) / r in the vertical equation) are dropped by advecting the
    horizontal velocity v_h = M / rho in the horizontal equation and w as a
    scalar in the vertical one. Returns (AC_h at the centres, AC_r at the
    interfaces)."""
    g, vg, pl, rhat = model.grid, model.vg, model.planet, model.rhat
    k = model.vorder
    vh = X.M / X.rho[..., None]
    w = Wc / X.rho
    A_h = np.zeros_like(X.M)
    for j in range(3):
        A_h[..., j] = op.div_h_levels(g, vg, X.M * vh[..., j:j + 1]) \
            + op.div_v(vg, X.W * op.interp_to_interfaces(vg, vh[..., j], k))
    A_r = op.div_h_levels(g, vg, X.M * w[..., None]) + op.div_v(vg, X.W * op.interp_to_interfaces(vg, w, k))
    f = 2.0 * pl.omega * rhat[:, 2]
    C_h = f[:, None, None] * np.cross(np.broadcast_to(rhat[:, None, :], X.M.shape), X.M)
    return op.project_h(rhat, A_h + C_h), op.interp_to_interfaces(vg, A_r, k)


def slow_terms(model, X, Kd):
    """Right-hand sides of Eqs. dens2, mom2, momr2 and pt2 at the stage state
    X = Phi^(s) (reading R1), plus the small-step coefficients."""
    g, vg, pl = model.grid, model.vg, model.planet
    rhat = model.rhat
    N, nv = X.rho.shape
    p = pressure(pl, X.Th)

    # full 3-D momentum and velocity at the centres (reading R6)
    Wc = op.interp_to_centres(vg, X.W, model.vorder)
    mom = X.M + Wc[..., None] * rhat[:, None, :]
    vel = mom / X.rho[..., None]

    if vg.shallow:
        AC_h, AC_r = _shallow_advection_coriolis(model, X, Wc)
    else:
        # advection A_j = div_h(M v_j) + r^-2 d(r^2 W v_j)/dr
        A = np.zeros((N, nv, 3))
        for j in range(3):
            A[..., j] = op.div_h_levels(g, vg, X.M * vel[..., j:j + 1]) \
                + op.div_v(vg, X.W * op.interp_to_interfaces(vg, vel[..., j], model.vorder))
        # Coriolis 2 Omega x (rho v), Omega along z
        Om = np.array([0.0, 0.0, pl.omega])
        C = 2.0 * np.cross(Om[None, None, :], mom)
        AC_h = op.project_h(rhat, A + C)
        AC_r = op.interp_to_interfaces(vg, op.radial(rhat, A + C), model.vorder)

    rho_i = op.interp_to_interfaces(vg, X.rho)

    if model.hyperdiffusion:
        F_rho, F_M, F_W, F_Th = hyperdiffusion(model, X, p, Kd)
    else:
        F_rho, F_M, F_W, F_Th = (np.zeros_like(X.rho), np.zeros_like(X.M),
                                 np.zeros_like(X.W), np.zeros_like(X.Th))

    S_M = op.project_h(rhat, -op.grad_h_levels(g, vg, p) - AC_h + F_M)
    if model.hydrostatic:
        S_W = -op.ddz_at_interfaces(vg, p) - pl.gravity * rho_i       # reading H1
    else:
        S_W = -op.ddz_at_interfaces(vg, p) - pl.gravity * rho_i - AC_r + F_W
    S_W[:, 0] = 0.0
    S_W[:, -1] = 0.0
    S_rho = -op.div_h_levels(g, vg, X.M) - op.div_v(vg, X.W) + F_rho
    S_Th = F_Th

    theta = X.Th / X.rho
    return dict(p=p, S_M=S_M, S_W=S_W, S_rho=S_rho, S_Th=S_Th, theta=theta,
                theta_i=op.interp_to_interfaces(vg, theta),
                Pi=pl.gamma * p / X.Th,
                # the parts, for the anelastic switch (oracle.anelastic)
                AC_h=AC_h, AC_r=AC_r, F_M=F_M, F_W=F_W)


# ----------------------------------------------------------- vertical solve

def vertical_matrices(vg):
    """Discrete vertical operators of one column as dense matrices acting on
    the interior interfaces (1..nv-1) or on the centres (0..nv-1):
    Dv (nv x nv-1) = r^-2 d(r^2 .)/dr restricted to the interior interfaces,
    Gz (nv-1 x nv) = d/dr from centres to interfaces,
    Iz (nv-1 x nv) = Lagrange k = 1 interpolation from centres to interfaces."""
    nv = vg.nv
    E = np.eye(nv + 1)[:, 1:-1]                       # interior interface basis
    Dv = op.div_v(vg, E.T).T                          # (nv, nv-1)
    Ec = np.eye(nv)
    Gz = op.ddz_at_interfaces(vg, Ec)[:, 1:-1].T      # (nv-1, nv)
    Iz = op.interp_to_interfaces(vg, Ec)[:, 1:-1].T   # (nv-1, nv)
    return Dv, Gz, Iz


def vertical_solve(model, dtau, Wstar, S_W, a, b, c, theta_i, Pi):
    """Reading R3. With
        rho*+ = a - dtau Dv W,   Th+ = b - dtau Dv diag(theta_i) W,
        p*+   = c - dtau diag(Pi) Dv diag(theta_i) W,
        W     = W* + dtau (S_W - Gz p*+ - g Iz rho*+)
    the unknown W (interior interfaces of every column) solves
        [I - dtau^2 Gz diag(Pi) Dtheta - dtau^2 g Iz Dv] W
            = W* + dtau S_W - dtau Gz c - dtau g Iz a,
    solved here with a dense batched LU (numpy.linalg.solve). Under the
    hydrostatic switch (reading H1) the identity and W* carry the factor
    delta = 0."""
    vg, pl = model.vg, model.planet
    delta = 0.0 if model.hydrostatic else 1.0
    nv = vg.nv
    Dv, Gz, Iz = vertical_matrices(vg)
    N = a.shape[0]
    th = theta_i[:, 1:-1]                              # (N, nv-1)
    Dth = Dv[None, :, :] * th[:, None, :]              # (N, nv, nv-1)
    GPi = Gz[None, :, :] * Pi[:, None, :]              # (N, nv-1, nv)
    A = delta * np.eye(nv - 1)[None] - dtau ** 2 * (GPi @ Dth) - dtau ** 2 * pl.gravity * (Iz @ Dv)[None]
    rhs = delta * Wstar[:, 1:-1] + dtau * S_W[:, 1:-1] - dtau * (c @ Gz.T) - dtau * pl.gravity * (a @ Iz.T)
    Wint = np.linalg.solve(A, rhs[..., None])[..., 0]
    W = np.zeros((N, nv + 1))
    W[:, 1:-1] = Wint
    return W


# ----------------------------------------------------------- small step

def divergence_damping(model, M, W, Kd):
    """Sec. 4, the divergence-damping terms of Eqs. diff_vx-vz (reading R5):
    D = div_h M + r^-2 d(r^2 W)/dr, the 3-D divergence of the momentum (M at
    the centres, W at the interfaces), and the damping -K_d grad_h(lap D),
    the horizontal gradient (Eq. grad, projected by Eq. proj_h) of the
    Sec. 4 Laplacian of D. On the sphere this equals the printed
    -K_d P_h lap(grad_h D) (the projected Cartesian Laplacian of a gradient
    field is the gradient of the Laplacian), and the discrete form is the
    more accurate of the two (reading R5)."""
    g, vg = model.grid, model.vg
    D = op.div_h_levels(g, vg, M) + op.div_v(vg, W)
    return -Kd * op.grad_h_levels(g, vg, op.lap_levels(g, vg, D))


def small_step(model, Xs, co, pert, dtau, Kd):
    """One forward-backward small step (Sec. 3), order of Sec. 3: horizontal
    momentum (explicit, Eq. mom2 with the divergence damping of Sec. 4), then
    vertical momentum (implicit, Eq. momr2), then density (Eq. dens2), then
    rho theta (Eq. pt2) and p* (Eq. theta_to_p)."""
    g, vg, pl = model.grid, model.vg, model.planet
    rhat = model.rhat
    rho_s, M_s, W_s, Th = pert["rho"], pert["M"], pert["W"], pert["Th"]
    p_s = pert["p"]

    # divergence damping (reading R5) of the total momentum
    DD = divergence_damping(model, Xs.M + M_s, Xs.W + W_s, Kd) if model.divergence_damping else 0.0

    # Eq. mom2 (explicit)
    M_new = op.project_h(rhat, M_s + dtau * (-op.grad_h_levels(g, vg, p_s) + DD + co["S_M"]))

    # Eqs. dens2 / pt2 with everything but the implicit vertical fluxes
    theta = co["theta"]
    a = rho_s + dtau * (co["S_rho"] - op.div_h_levels(g, vg, M_new))
    Mtot = Xs.M + M_new
    b = Th + dtau * (co["S_Th"] - op.div_h_levels(g, vg, theta[..., None] * Mtot)
                     - op.div_v(vg, co["theta_i"] * Xs.W))
    c = p_s + co["Pi"] * (b - Th)

    # Eq. momr2 (implicit, reading R3)
    W_new = vertical_solve(model, dtau, W_s, co["S_W"], a, b, c, co["theta_i"], co["Pi"])

    # Eq. dens2 and Eq. pt2 with the new vertical momentum
    rho_new = a - dtau * op.div_v(vg, W_new)
    Th_new = b - dtau * op.div_v(vg, co["theta_i"] * W_new)
    # Eq. theta_to_p
    p_new = pressure(pl, Th_new) - co["p"]
    return dict(rho=rho_new, M=M_new, W=W_new, Th=Th_new, p=p_new)


# ----------------------------------------------------------- large step

def stage_schedule(dt, n_small):
    """Sec. 3 (Wicker-Skamarock RK3 with the Klemp small-step counts):
    (dtau, number of small steps) for the three stages."""
    if n_small < 2 or n_small % 2:
        raise ValueError("n_small must be even and >= 2")
    return [(dt / 3.0, 1), (dt / n_small, n_small // 2), (dt / n_small, n_small)]


def rk_stage(model, Xt, Xs, dtau, nsub, Kd):
    """One RK3 stage (reading R1): the slow terms at the stage state Xs, the
    perturbations started at Xt - Xs (p* from Eq. theta_to_p), nsub small
    steps of dtau, and the stage's result X^(s+1) = Xs + X*."""
    co = slow_terms(model, Xs, Kd)
    pert = dict(rho=Xt.rho - Xs.rho, M=Xt.M - Xs.M, W=Xt.W - Xs.W, Th=Xt.Th.copy(),
                p=pressure(model.planet, Xt.Th) - co["p"])
    for _ in range(nsub):
        pert = small_step(model, Xs, co, pert, dtau, Kd)
    return State(Xs.rho + pert["rho"], Xs.M + pert["M"], Xs.W + pert["W"], pert["Th"])


def large_step(model, X, dt, n_small, energy_fixer=False, budget=None):
    """One large step: three RK3 stages of small steps (reading R1), then, if
    energy_fixer, the uniform internal-energy adjustment of energy.energy_fix
    (Sec. 3), then the physics of Sec. 5. If budget is a list, the step's
    budget row (energy.budget_row) is appended to it."""
    from .physics import apply_physics
    if model.anelastic:
        from .anelastic import large_step as anelastic_large_step
        return anelastic_large_step(model, X, dt)
    Kd = model.Kd(dt)
    Xt = X
    Xs = X
    for dtau, nsub in stage_schedule(dt, n_small):
        Xs = rk_stage(model, Xt, Xs, dtau, nsub, Kd)
    if energy_fixer or budget is not None:
        from .energy import budget_row, energy_fix
        Xd, dT = Xs, 0.0
        if energy_fixer:
            Xs, dT = energy_fix(model, Xt, Xd)
        if budget is not None:
            budget.append(budget_row(model, Xt, Xd, dT))
    return apply_physics(model, Xs, dt)


def run(model, X, n_large, n_small, dt, energy_fixer=False, budget=None):
    for _ in range(n_large):
        X = large_step(model, X, dt, n_small, energy_fixer, budget)
    return X


# ----------------------------------------------------------- initial state

def hydrostatic_profile(model, T, p_surf):
    """Discretely balanced column for the layer temperatures T (nv,):
    (p_i - p_i-1)/dz + g rho_iface = 0 at every interior interface, with
    rho = p/(Rd T) and rho_iface the Lagrange k = 1 interpolation, so that
    the slow vertical force of Eq. momr2 vanishes at rest. The lowest centre
    is p_surf exp(-g z_0 / (Rd T_0)) (hydrostatic at constant T)."""
    vg, pl = model.vg, model.planet
    nv = vg.nv
    p = np.zeros(nv)
    p[0] = p_surf * np.exp(-pl.gravity * vg.zc[0] / (pl.Rd * T[0]))
    for i in range(1, nv):
        z0, z1, zh = vg.zc[i - 1], vg.zc[i], vg.zi[i]
        w0 = (zh - z1) / (z0 - z1)
        w1 = (zh - z0) / (z1 - z0)
        dz = z1 - z0
        p[i] = p[i - 1] * (1.0 - pl.gravity * dz * w0 / (pl.Rd * T[i - 1])) \
            / (1.0 + pl.gravity * dz * w1 / (pl.Rd * T[i]))
    return p


def held_suarez_start_profile(model, p_surf, tol=1e-12, max_iter=1000):
    """The layer temperatures of the Held-Suarez start of Sec. 6.1: every
    column at rest with the T_eq of Sec. 6.1 at the equator, in hydrostatic
    equilibrium. T_eq depends on p and the balanced p on T, so the column is
    the fixed point T = T_eq(p(T)) with p(T) = hydrostatic_profile, iterated
    from 315 K until no layer moves by more than tol K. Returns (T, p)."""
    from .physics import held_suarez_coefficients
    nv = model.vg.nv
    T = np.full(nv, 315.0)
    for _ in range(max_iter):
        p = hydrostatic_profile(model, T, p_surf)
        T_new = held_suarez_coefficients(np.ones(nv), p, np.zeros(nv), model.planet.kappa)[2]
        done = np.abs(T_new - T).max() <= tol
        T = T_new
        if done:
            return T, hydrostatic_profile(model, T, p_surf)
    raise RuntimeError("the Held-Suarez start profile did not converge")


def initial_state(model, T0, p_surf, noise_amp=0.0, u=None, profile=None):
    """Isothermal atmosphere at rest in discrete hydrostatic balance (Sec. 6
    starts both benchmarks at rest in hydrostatic equilibrium). With
    ``noise_amp`` > 0 the temperature gets amp (2u - 1) at fixed pressure, so
    the perturbation is carried by the density; ``u`` (N, nv) in [0, 1) are
    the random numbers, passed in. profile="held_suarez": the layer
    temperatures of held_suarez_start_profile instead of T0."""
    pl = model.planet
    N, nv = model.grid.ncol, model.vg.nv
    if profile == "held_suarez":
        T1, p1 = held_suarez_start_profile(model, p_surf)
    else:
        T1 = np.full(nv, float(T0))
        p1 = hydrostatic_profile(model, T1, p_surf)
    p = np.broadcast_to(p1, (N, nv)).copy()
    T = np.broadcast_to(T1, (N, nv)).copy()
    if noise_amp > 0.0:
        T = T + noise_amp * (2.0 * u - 1.0)
    rho = p / (pl.Rd * T)
    return State(rho, np.zeros((N, nv, 3)), np.zeros((N, nv + 1)), rhotheta_from_p(pl, p))
