"""Oracle anelastic switch (Sec. 3, list of approximations), float64, numpy
and scipy.sparse.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3 describes the anelastic approximation in one sentence: the density
in the divergence term of the mass continuity equation is replaced by a
reference density that depends on altitude only, after Ogura and Phillips
(1962), to neglect the elasticity of the fluid and so filter sound waves.
The paper gives no formulation beyond that. Readings:

A-1 Continuity becomes the constraint div(rho0 v) = 0: the density tendency
    is dropped with the elasticity (that is what removes the sound waves) and
    rho0(z) is the reference column (the resting, discretely balanced start
    column). The state keeps rho = rho0, M = rho0 v_h at the centres and
    W = rho0_i v_r at the interfaces, so the constraint is the discrete 3-D
    divergence of Sec. 2.2 / Sec. 3, D(M, W) = div_h M + r^-2 d(r^2 W)/dr = 0.
A-2 Momentum: the pressure force becomes -grad p' with p' the pressure that
    enforces the constraint; the gravity and the hydrostatic part of the
    pressure leave the buoyancy of Ogura and Phillips, b = g rho0 theta' /
    theta0 (theta' = theta - theta0, Th = rho0 theta), at the interfaces with
    rho0 and theta' / theta0 interpolated linearly. Advection, Coriolis and
    hyperdiffusion are those of the compressible model (Sec. 3-4) at the
    anelastic state.
A-3 Entropy: rho theta in flux form, dTh/dt = -div_h(theta M) - div_v(theta_i W)
    + F_Th, with the hyperdiffusion of Sec. 4.
A-4 Time stepping: with no acoustic terms the split-explicit small steps go;
    each of the three RK3 stages (dt/3, dt/2, dt, the stage lengths of
    Sec. 3) is one projection step from X^t: M^ = M^t + dt_s S_M(X^(s)),
    W^ = W^t + dt_s S_W(X^(s)), then p' from L p' = D(M^, W^) / dt_s with
    L = D o G (G the gradient of Eq. grad per level and d/dr between the
    centres, zero normal flow at the ground and the lid), M = M^ - dt_s G_h p',
    W = W^ - dt_s G_v p'; Th^(s+1) = Th^t + dt_s S_Th(X^(s)). The constant of
    p' is fixed by a zero volume mean.
A-5 The solve is direct (a sparse LU, scipy.sparse.linalg.splu, with three
    steps of iterative refinement) on the operator built column by column
    from the oracle's own grad_h and div_h, bordered by the volume-mean
    condition (L is singular: constants are its null
    space, and the volumes its left null vector, which the right-hand side
    meets by the exact discrete Gauss theorem).
A-6 Physics (Sec. 5-6) as in the compressible model, at rho = rho0.
"""

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import dycore as dc
from . import operators as op


def reference_column(model, T0, p_surf, profile=None):
    """(rho0, theta0) of the resting start column (dycore.initial_state
    without noise): the anelastic reference."""
    X = dc.initial_state(model, T0, p_surf, profile=profile)
    return X.rho[0].copy(), X.Th[0] / X.rho[0]


def anelastic_start(model, T0, p_surf, theta_prime=None, profile=None):
    """The anelastic state at rest on the reference column, with an optional
    theta' (N, nv) added: rho = rho0, M = W = 0, Th = rho0 (theta0 + theta')."""
    rho0, theta0 = reference_column(model, T0, p_surf, profile)
    model.reference = (rho0, theta0)
    N, nv = model.grid.ncol, model.vg.nv
    th = np.broadcast_to(theta0, (N, nv)).copy()
    if theta_prime is not None:
        th = th + theta_prime
    rho = np.broadcast_to(rho0, (N, nv)).copy()
    return dc.State(rho, np.zeros((N, nv, 3)), np.zeros((N, nv + 1)), rho * th)


def divergence(model, M, W):
    """The discrete 3-D divergence of the momentum, D(M, W) at the centres."""
    return op.div_h_levels(model.grid, model.vg, M) + op.div_v(model.vg, W)


def grad_v(vg, phi):
    """d phi / dr at the interior interfaces (zero at the ground and the lid)."""
    return op.ddz_at_interfaces(vg, phi)


def horizontal_operator(grid):
    """D_h o G_h on the unit sphere as a sparse (N, N) matrix, column j the
    divergence of the gradient of the unit field e_j."""
    E = np.eye(grid.ncol)
    A = op.div_h(grid, op.grad_h(grid, E))            # (N, N): row i, unit field j
    A[np.abs(A) < 1e-300] = 0.0
    return sps.csr_matrix(A)


def vertical_operator(vg):
    """div_v o grad_v on one column, (nv, nv)."""
    return op.div_v(vg, grad_v(vg, np.eye(vg.nv))).T


def operator(model):
    """The 3-D operator L = D o G on all cells, unknown index c * nv + k."""
    if getattr(model, "_anelastic_L", None) is None:
        vg = model.vg
        Lh = horizontal_operator(model.grid)
        Lv = sps.csr_matrix(vertical_operator(vg))
        L = sps.kron(Lh, sps.diags(1.0 / vg.rc ** 2)) + sps.kron(sps.identity(model.grid.ncol), Lv)
        model._anelastic_L = L.tocsr()
    return model._anelastic_L


def volumes(model):
    return model.grid.area[:, None] * model.vg.rc[None, :] ** 2 * model.vg.dz[None, :]


def pressure(model, rhs):
    """p' with L p' = rhs and zero volume mean (reading A-5)."""
    L = operator(model)
    v = volumes(model).ravel()
    n = L.shape[0]
    # the border scaled to the size of L's entries (the volumes are ~1e16 m^3)
    s = abs(L).sum() / L.nnz
    col = sps.csr_matrix(np.full((n, 1), s))
    row = sps.csr_matrix((s * v / v.mean())[None, :])
    B = sps.bmat([[L, col], [row, None]]).tocsc()
    lu = spla.splu(B)
    b = np.concatenate([rhs.ravel(), [0.0]])
    x = lu.solve(b)
    for _ in range(3):                    # iterative refinement against the LU's rounding
        x = x + lu.solve(b - B @ x)
    return x[:n].reshape(rhs.shape)


def project(model, Mh, Wh, dts):
    """Reading A-4: the momentum (Mh, Wh) made divergence-free by the pressure
    p' of L p' = D(Mh, Wh) / dts. Returns (M, W, p')."""
    g, vg = model.grid, model.vg
    phi = pressure(model, divergence(model, Mh, Wh) / dts)
    M = Mh - dts * op.grad_h_levels(g, vg, phi)
    W = Wh - dts * grad_v(vg, phi)
    return M, W, phi


def slow_terms(model, X, Kd):
    """S_M, S_W and S_Th of readings A-2 and A-3 at the anelastic state X."""
    g, vg, pl = model.grid, model.vg, model.planet
    rho0, theta0 = model.reference
    co = dc.slow_terms(model, X, Kd)
    S_M = op.project_h(model.rhat, -co["AC_h"] + co["F_M"])
    ratio = (X.Th / X.rho - theta0[None, :]) / theta0[None, :]           # theta' / theta0
    b = pl.gravity * op.interp_to_interfaces(vg, np.broadcast_to(rho0, X.rho.shape)) \
        * op.interp_to_interfaces(vg, ratio)
    if model.hydrostatic:
        raise ValueError("the anelastic switch keeps the vertical momentum's inertia")
    S_W = b - co["AC_r"] + co["F_W"]
    S_W[:, 0] = 0.0
    S_W[:, -1] = 0.0
    theta = co["theta"]
    S_Th = co["S_Th"] - op.div_h_levels(g, vg, theta[..., None] * X.M) - op.div_v(vg, co["theta_i"] * X.W)
    return S_M, S_W, S_Th


def large_step(model, X, dt):
    """One large step of the anelastic model (readings A-1..A-6)."""
    from .physics import apply_physics
    Kd = model.Kd(dt)
    Xt = X
    Xs = X
    for dts in (dt / 3.0, dt / 2.0, dt):
        S_M, S_W, S_Th = slow_terms(model, Xs, Kd)
        M, W, _ = project(model, Xt.M + dts * S_M, Xt.W + dts * S_W, dts)
        Xs = dc.State(Xt.rho.copy(), M, W, Xt.Th + dts * S_Th)
    return apply_physics(model, Xs, dt)
