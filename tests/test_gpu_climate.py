"""Zonal band means on the GPU (thor_zonal_accumulate / thor_zonal_read)
against the oracle's (oracle/climate.py) on the same state, and the climate
runner on a short run."""

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
