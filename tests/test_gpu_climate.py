"""Zonal band means and the per-cell time mean of w on the GPU
(thor_zonal_accumulate / thor_zonal_read / thor_zonal_read_w) against the
oracle's (oracle/climate.py) on the same states, and the climate runner on
short runs."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from harness import Pair
from oracle import climate as ocl
import workloads as wls

SMALL = wls.HS_G4.with_(name="hs_g3_L12", glevel=3, nv=12, n_large=3)


@pytest.mark.parametrize("precision,nlat", [(thor.THOR_FP64, 12), (thor.THOR_MIXED, 18)])
def test_zonal_means_match_the_oracle(precision, nlat):
    p = Pair(SMALL, precision=precision)
    try:
        thor.thor_step(p.state, SMALL.n_large, SMALL.n_small, SMALL.dt)
        thor.thor_zonal_accumulate(p.state, nlat)
        got, n = thor.thor_zonal_read(p.state, nlat, SMALL.nv)
        assert n == 1
        ref = ocl.zonal_band_means(p.model, p.get(), nlat)   # the library's own state, in float64
        assert np.abs(ref[..., 1]).max() > 1e-3              # there is wind
        np.testing.assert_allclose(got[..., 0], ref[..., 0], rtol=1e-12)
        for q in range(1, 9):
            scale = np.abs(ref[..., q]).max() + 1e-300
            assert np.abs(got[..., q] - ref[..., q]).max() <= 1e-9 * scale, (ocl.QUANTITIES[q],)
    finally:
        p.close()


def test_accumulate_read_and_reset():
    p = Pair(SMALL, precision=thor.THOR_MIXED)
    try:
        thor.thor_step(p.state, 1, SMALL.n_small, SMALL.dt)
        thor.thor_zonal_accumulate(p.state, 9)
        one, n1 = thor.thor_zonal_read(p.state, 9, SMALL.nv)
        thor.thor_zonal_accumulate(p.state, 9)
        two, n2 = thor.thor_zonal_read(p.state, 9, SMALL.nv, reset=True)
        assert (n1, n2) == (1, 2)
        # the same state twice: twice the first read, up to the order of the
        # float64 atomic additions of the band sums (amplified in the
        # covariances, differences of nearly equal products such as [vT] and
        # [v][T])
        for q in range(9):
            scale = np.abs(one[..., q]).max() + 1e-300
            assert np.abs(two[..., q] - 2 * one[..., q]).max() <= (1e-14 if q < 5 else 1e-10) * scale, q
        zero, n0 = thor.thor_zonal_read(p.state, 9, SMALL.nv)
        assert n0 == 0 and not zero.any()
        other, n = thor.thor_zonal_read(p.state, 7, SMALL.nv)     # never accumulated
        assert n == 0 and not other.any()
        with pytest.raises(thor.ThorError):
            thor.thor_zonal_accumulate(p.state, 0)
    finally:
        p.close()


def test_climate_runner_short_held_suarez():
    """Twenty days of Held-Suarez at glevel 3 x 12 levels (mixed precision):
    the runner accumulates daily samples and the summary is finite; the
    forcing has started the mid-latitude westerlies (positive zonal wind
    aloft in both hemispheres)."""
    from paper_1607_05535_gb300 import climate
    means, samples, seconds, diag = climate.run(thor, glevel=3, nv=12, z_top=32.0e3, dt=1800.0, n_small=6,
                                                days=20.0, spinup_days=10.0, nlat=12)
    assert samples == 10 and diag["nonfinite"] == 0
    s = climate.summarize(means, wls.EARTH.radius, wls.EARTH.gravity)
    assert np.all(np.isfinite(means))
    assert s["jets"]["north"]["u_ms"] > 0 and s["jets"]["south"]["u_ms"] > 0


@pytest.mark.parametrize("precision", [thor.THOR_FP64, thor.THOR_MIXED])
def test_time_mean_w_and_imprint_map_match_the_oracle(precision):
    """The per-cell time mean [w] that thor_zonal_accumulate keeps, over four
    states, against the oracle's w of the library's own states averaged on
    the host, and the [w*] map built from it; thor_zonal_read's reset clears
    it."""
    from paper_1607_05535_gb300 import climate
    nlat = 12
    p = Pair(SMALL, precision=precision)
    try:
        ws = []
        for _ in range(4):
            thor.thor_step(p.state, 1, SMALL.n_small, SMALL.dt)
            thor.thor_zonal_accumulate(p.state, nlat)
            ws.append(ocl.cell_w(p.model, p.get()))
        got_lib, n = thor.thor_zonal_read_w(p.state, nlat, p.ncol, p.nv)
        assert n == 4
        got = np.empty_like(got_lib)
        got[p.perm] = got_lib
        ref = np.mean(ws, axis=0)
        assert np.abs(ref).max() > 1e-6                                # the air moves vertically
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        pts = np.empty((p.ncol, 3))
        pts[p.perm] = thor.thor_grid_points(p.grid)
        area = np.empty(p.ncol)
        area[p.perm] = thor.thor_grid_areas(p.grid)
        np.testing.assert_allclose(climate.w_star(got, pts, area, nlat), ocl.w_star(p.model, ref, nlat),
                                   atol=1e-11 * np.abs(ref).max())
        thor.thor_zonal_read(p.state, nlat, p.nv, reset=True)
        zero, n0 = thor.thor_zonal_read_w(p.state, nlat, p.ncol, p.nv)
        assert n0 == 0 and not zero.any()
        thor.thor_zonal_accumulate(p.state, nlat)
        one, n1 = thor.thor_zonal_read_w(p.state, nlat, p.ncol, p.nv)
        assert n1 == 1 and np.abs(one).max() > 0
    finally:
        p.close()


def test_climate_runner_switches_and_post_processing():
    """Ten days of Held-Suarez at glevel 3 with both approximation switches:
    the runner's extras, [w*] summary and pressure-level fields are finite."""
    from paper_1607_05535_gb300 import climate
    extras = {}
    means, samples, seconds, diag = climate.run(thor, glevel=3, nv=12, z_top=32.0e3, dt=1800.0, n_small=6,
                                                days=10.0, spinup_days=5.0, nlat=12, shallow=True,
                                                hydrostatic=True, extras=extras)
    assert samples == 5 and diag["nonfinite"] == 0
    ws = climate.w_star(extras["w_mean"], extras["points"], extras["areas"], 12)
    imp = climate.imprint_summary(ws, extras["w_mean"], extras["points"], extras["areas"], 12)
    assert np.isfinite(list(imp.values())).all() and 0 <= imp["w_star_wave5_share"] <= 1
    pm = means[..., 4]
    s = climate.summarize(means, wls.EARTH.radius, wls.EARTH.gravity, np.geomspace(pm.max(), pm.min(), 8))
    assert s["u_p_levels"][0][0] is not None or s["u_p_levels"][1][0] is not None
