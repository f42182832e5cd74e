"""libthor loads, exports every entry point of include/thor.h, rejects bad
arguments, and its host grid builder agrees with the oracle. No GPU compute."""

import ctypes
import os
import re

import numpy as np
import pytest
from scipy.spatial import cKDTree

from conftest import ROOT, oracle_grid

thor = pytest.importorskip("paper_1607_05535_gb300")


def test_exports_match_header():
    hdr = open(os.path.join(ROOT, "include", "thor.h")).read()
    declared = set(re.findall(r"\b(thor_[a-z_]+)\s*\(", hdr))
    lib = ctypes.CDLL(thor.LIBRARY_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(thor.EXPORTED)


def test_invalid_arguments():
    with pytest.raises(thor.ThorError) as e:
        thor.thor_grid_create(11, 4, 6.4e6, 3e4)
    assert e.value.status == thor.THOR_EINVAL
    for args in ((3, 1, 6.4e6, 3e4), (3, 4, -1.0, 3e4), (3, 4, 6.4e6, 0.0), (-1, 4, 6.4e6, 3e4)):
        with pytest.raises(thor.ThorError):
            thor.thor_grid_create(*args)
    assert thor.thor_strerror(thor.THOR_ETIMEOUT) == "device wait timed out"


def test_state_init_argument_checks_need_no_device():
    """thor_state_init refuses a bad start (unknown profile, T0 <= 0 for the
    isothermal profile, a planet radius other than the grid's) on the host,
    before any CUDA call."""
    grid = thor.thor_grid_create(2, 4, 6.4e6, 3e4, thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, 5))
    try:
        planet = thor.thor_planet(6.4e6, 7.292e-5, 9.8, 287.0, 1005.0, 1.0e5, 0.0)
        for kw in (dict(profile=2), dict(profile=-1), dict(T0=0.0), dict(T0=-5.0, profile=0)):
            a = dict(T0=300.0, profile=0)
            a.update(kw)
            init = thor.thor_init(a["T0"], 1.0e5, 0.0, 1, 0, 300.0, thor.THOR_FP64, 1, 1, 0, 0, a["profile"])
            with pytest.raises(thor.ThorError) as e:
                thor.thor_state_init(grid, planet, init)
            assert e.value.status == thor.THOR_EINVAL, kw
        bad = thor.thor_planet(6.5e6, 7.292e-5, 9.8, 287.0, 1005.0, 1.0e5, 0.0)
        init = thor.thor_init(300.0, 1.0e5, 0.0, 1, 0, 300.0, thor.THOR_FP64, 1, 1, 0, 0, 0)
        with pytest.raises(thor.ThorError) as e:
            thor.thor_state_init(grid, bad, init)
        assert e.value.status == thor.THOR_EINVAL
    finally:
        thor.thor_grid_destroy(grid)


def test_ensemble_argument_checks_need_no_device():
    """Argument errors of the ensemble and autotuner entry points are caught
    on the host, before any CUDA call."""
    for members in ([], [None]):
        with pytest.raises(thor.ThorError) as e:
            thor.thor_ensemble_create(members)
        assert e.value.status == thor.THOR_EINVAL
    with pytest.raises(thor.ThorError) as e:
        thor.thor_ensemble_create([None] * (thor.THOR_ENSEMBLE_MAX + 1))
    assert e.value.status == thor.THOR_EINVAL
    for call in (lambda: thor.thor_ensemble_step(None, 1, [8], [600.0]),
                 lambda: thor.thor_ensemble_tune(None, thor.THOR_TUNE_BLOCK, 128),
                 lambda: thor.thor_ensemble_info(None),
                 lambda: thor.thor_autotune(None, 8, 600.0),
                 lambda: thor.thor_ensemble_autotune(None, [8], [600.0])):
        with pytest.raises(thor.ThorError) as e:
            call()
        assert e.value.status == thor.THOR_EINVAL
    thor.thor_ensemble_destroy(None)
    for limit in (0, 2000001):
        with pytest.raises(thor.ThorError) as e:
            thor.thor_wait_selftest(0, limit)
        assert e.value.status == thor.THOR_EINVAL
    with pytest.raises(thor.ThorError) as e:
        thor.thor_budget_read(None)
    assert e.value.status == thor.THOR_EINVAL
    for knob in (thor.THOR_TUNE_ENERGY_FIXER, thor.THOR_TUNE_BUDGET):
        with pytest.raises(thor.ThorError) as e:
            thor.thor_tune(None, knob, 1)
        assert e.value.status == thor.THOR_EINVAL


def _match(P, O):
    d, idx = cKDTree(O.points).query(P)
    assert len(np.unique(idx)) == len(idx)
    return d, idx


@pytest.mark.parametrize("g, max_iter, tol", [(0, 10, 0.0), (2, 10, 0.0), (4, 10, 0.0), (3, 100000, 1e-5),
                                            (6, 10, 0.0)])
def test_grid_parity_with_oracle(g, max_iter, tol):
    """Independent builders (rhombus lattice vs. triangle list) give the same
    points, neighbour sets, areas and spring iteration count."""
    sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, tol, max_iter)
    G = thor.thor_grid_create(g, 4, 6.371e6, 3.0e4, sp)
    try:
        info = thor.thor_grid_info(G)
        P = thor.thor_grid_points(G)
        A = thor.thor_grid_areas(G)
        nb = thor.thor_grid_neighbours(G)
    finally:
        thor.thor_grid_destroy(G)
    O = oracle_grid(g, max_iter=max_iter, tol=tol)
    assert info["ncol"] == O.ncol == 10 * 4 ** g + 2 and info["npent"] == 12
    assert info["spring_iters"] == O.spring_iters
    assert info["spring_converged"] == O.spring_converged
    d, idx = _match(P, O)
    assert d.max() < 1e-12
    assert np.max(np.abs(A - O.area[idx])) < 1e-13
    for c in range(len(P)):
        mine = {idx[x] for x in nb[c] if x >= 0}
        assert mine == set(O.nbr[idx[c], :O.nn[idx[c]]].tolist())


def test_canonical_numbering():
    """Columns are numbered rhombus by rhombus, then the two poles."""
    G = thor.thor_grid_create(2, 4, 1.0, 0.1, thor.thor_spring(1.15, 1, 1, 0.01, 0.0, 0))
    P = thor.thor_grid_points(G)
    thor.thor_grid_destroy(G)
    assert np.allclose(P[-2], [0, 0, 1]) and np.allclose(P[-1], [0, 0, -1])
    n = 4
    # north rhombus 0 owns U_0 (lat atan(1/2), lon 0) at its lattice origin
    lat = np.arctan(0.5)
    assert np.allclose(P[0], [np.cos(lat), 0, np.sin(lat)])
    # south rhombus 0 owns L_0 (lat -atan(1/2), lon 36 deg)
    assert np.allclose(P[5 * n * n], [np.cos(lat) * np.cos(np.pi / 5), np.cos(lat) * np.sin(np.pi / 5), -np.sin(lat)])


@pytest.mark.parametrize("gf,gc,iters", [(3, 2, 10), (4, 3, 10), (5, 4, 0), (4, 2, 10)])
def test_coarse_map_is_the_nearest_centre(gf, gc, iters):
    """thor_grid_coarse_map (the closure's coarse-graining map, built on the
    host by a walk over the coarse neighbour graph) gives every fine column
    the coarse column of largest dot product, as a brute-force search does;
    every coarse column receives at least one fine column."""
    sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, iters)
    F = thor.thor_grid_create(gf, 4, 6.371e6, 3.0e4, sp)
    C = thor.thor_grid_create(gc, 4, 6.371e6, 3.0e4, sp)
    try:
        m = thor.thor_grid_coarse_map(F, C)
        pf, pc = thor.thor_grid_points(F), thor.thor_grid_points(C)
        d = pf @ pc.T
        best = d.max(axis=1)
        assert np.all(d[np.arange(len(m)), m] >= best - 1e-15)
        assert len(np.unique(m)) == len(pc)
        with pytest.raises(thor.ThorError):
            thor._check(thor._lib.thor_grid_coarse_map(F, C, thor._ptr(m), len(m) - 1), "thor_grid_coarse_map")
    finally:
        thor.thor_grid_destroy(F)
        thor.thor_grid_destroy(C)
