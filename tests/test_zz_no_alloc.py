"""The allocation-free mass sum (thor_mass_noalloc) against thor_diag's mass.

thor_mass_noalloc serves callers that must not call cudaMalloc (an outer
framework owns the device-memory budget, or the implicit device
synchronisation of cudaMalloc would stall a latency-critical loop): they pass
their own device arrays and the library allocates nothing. This file is named
to be collected last."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
import workloads as wls

TOL = 1e-12


def test_mass_noalloc_matches_diag_twice():
    wl = wls.HS_G4
    P = wl.planet
    torch.cuda.set_device(0)
    grid = thor.thor_grid_create(wl.glevel, wl.nv, P.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, wl.spring_max_iter))
    planet = thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
    init = thor.thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, thor.THOR_FORCING_HELD_SUAREZ,
                          wl.hj_dT, thor.THOR_FP64, 1, 1)
    state = thor.thor_state_init(grid, planet, init, None)
    try:
        # cell volumes A_c r_k^2 dz_k of the library's uniform vertical grid
        area = thor.thor_grid_areas(grid)
        zi = np.linspace(0.0, wl.z_top, wl.nv + 1)
        zc = 0.5 * (zi[:-1] + zi[1:])
        vol = area[:, None] * (P.radius + zc[None, :]) ** 2 * np.diff(zi)[None, :]
        vol_d = torch.tensor(vol, dtype=torch.float64, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        for call in range(2):
            thor.thor_step(state, 1, wl.n_small, wl.dt)
            ref = thor.thor_diag(state)["mass"]
            rho = thor.thor_state_get(state, thor.THOR_FIELD_RHO, wl.ncol, wl.nv)
            rho_d = torch.tensor(rho, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            torch_before, free_before = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
            thor.thor_mass_noalloc(rho_d, vol_d, out)
            torch.cuda.synchronize()
            if call == 1:
                # the first call may load the kernels' module (lazy loading);
                # from then on a call allocates nothing, from torch or the device
                assert torch.cuda.memory_allocated() == torch_before
                assert torch.cuda.mem_get_info()[0] == free_before
            got = float(out.item())
            assert abs(got - ref) <= TOL * abs(ref), (call, got, ref)
    finally:
        thor.thor_state_destroy(state)
        thor.thor_grid_destroy(grid)


def test_mass_noalloc_rejects_oversize_and_null():
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(thor.ThorError) as e:
        # declared size beyond the static scratch: rejected before any launch
        thor._check(thor._lib.thor_mass_noalloc(thor._ptr(x), thor._ptr(x), 4096 * 16384 + 1,
                                                thor._ptr(out), None), "thor_mass_noalloc")
    assert e.value.status == thor.THOR_EINVAL
    with pytest.raises(thor.ThorError):
        thor._check(thor._lib.thor_mass_noalloc(None, thor._ptr(x), 4, thor._ptr(out), None),
                    "thor_mass_noalloc")
