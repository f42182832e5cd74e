"""Plain FP64 CPU oracle for the THOR dynamical core (Mendonca et al. 2016).

TEST INFRASTRUCTURE ONLY. This package is a slow, literal restatement of the
paper's discretisation in numpy float64, used to check the CUDA path. Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. The product path (``paper_1607_05535_gb300``)
never imports, links or calls anything here, and this package imports nothing
from the product.

Modules
-------
grid        Sec. 2: recursive icosahedron, spring dynamics (Eqs. spring_force,
            spr_vel, dbar), centroid relocation, metric terms.
operators   Sec. 2 / Sec. 3: Eqs. int_grid, flx_div, div_gauss, grad, the
            Laplacian of Sec. 4, the Lagrange vertical interpolation, the deep
            3-D operator split and Eqs. proj_h / proj_r.
dycore      Sec. 3-4: flux-form Euler equations (Eqs. mass, mom, entropy,
            pressure), the Wicker-Skamarock RK3 large step, the forward-backward
            small step (Eqs. dens2, mom2, momr2, pt2, theta_to_p) with the HE-VI
            vertical solve, hyperdiffusion and divergence damping (Eqs.
            diff_rho ... diff_p, kd, tau_d); the shallow-atmosphere and
            hydrostatic switches of Sec. 3; the resting starts of Sec. 6
            (isothermal, or the equatorial Held-Suarez T_eq in balance).
physics     Sec. 5-6: Eqs. im_eq_v, im_eq_t with the Held-Suarez (Eq.
            im_eq_fv and T_eq, K_T) and hot-Jupiter (Eqs. teq-hj, btrop, tvert)
            forcings.
diagnostics Global mass, energy, axial angular momentum and extrema (Sec. 3).
climate     Sec. 6.1: zonal band means of wind, temperature and pressure and
            the eddy covariances [u'v'], [v'T'] of one state; the
            grid-imprinting map [w*]; interpolation to pressure levels (Sec. 6).
energy      Sec. 3: the globally uniform internal-energy adjustment after
            Williamson (2009) and the per-step mass, energy and angular
            momentum budget.

Every reading of a passage that the paper leaves silent, ambiguous or garbled
is stated at the function that takes it.
"""
