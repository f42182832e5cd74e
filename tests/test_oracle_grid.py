"""Pins of the oracle grid (Sec. 2) against closed forms, invariants and the
paper's worked example. CPU only."""

import json
import os

import numpy as np
import pytest

from conftest import oracle_grid
from oracle import grid as og

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("g", [0, 1, 2, 3, 4])
def test_counts_and_euler(g):
    """Eq. grid_qts: N = 2 + 10 * 4^g; twelve pentagons; V - E + F = 2."""
    G = oracle_grid(g, modified=False)
    N = 2 + 10 * 4 ** g
    assert G.ncol == N
    assert np.count_nonzero(G.nn == 5) == 12
    assert np.count_nonzero(G.nn == 6) == N - 12
    F = len(G.faces)
    E = int(np.sum(G.nn)) // 2
    assert F == 20 * 4 ** g and E == 30 * 4 ** g
    assert N - E + F == 2


def test_worked_example():
    gold = json.load(open(os.path.join(GOLDEN, "grid_resolution.json")))
    n, dbar, th = og.mean_resolution(gold["glevel"], gold["radius_m"])
    assert n == gold["n_vertices_g5"]
    assert abs(dbar / 1e3 - gold["dbar_km"]) / gold["dbar_km"] < gold["dbar_rel_tol"]
    assert abs(np.degrees(th) - gold["theta_deg"]) < gold["theta_abs_tol_deg"]
    assert oracle_grid(5, modified=False).ncol == gold["n_vertices_g5"]


@pytest.mark.parametrize("modified", [False, True])
def test_areas_tile_the_sphere(modified):
    G = oracle_grid(3, modified=modified)
    assert abs(G.area.sum() - 4 * np.pi) < 1e-12
    assert abs(G.tri_area.sum() - 4 * np.pi) < 1e-12
    assert np.all(G.area > 0)


def test_edges_shared_antisymmetric():
    """Every control-volume edge is shared by exactly two cells with the same
    length and opposite normals (what makes Eq. div_gauss conservative)."""
    G = oracle_grid(3)
    seen = {}
    for i in range(G.ncol):
        m = G.nn[i]
        for k in range(m):
            j = G.nbr[i, (k + 1) % m]
            seen[(i, j)] = (G.edge_l[i, k], G.edge_n[i, k])
    for (i, j), (l, n) in seen.items():
        l2, n2 = seen[(j, i)]
        assert abs(l - l2) < 1e-15
        assert np.max(np.abs(n + n2)) < 1e-15


def test_rings_counter_clockwise():
    G = oracle_grid(3)
    P = G.points
    idx = np.arange(G.ncol)
    for k in range(6):
        a = P[G.nbr[idx, k % G.nn]] - P
        b = P[G.nbr[idx, (k + 1) % G.nn]] - P
        assert np.all(np.sum(np.cross(a, b) * P, axis=1) > 0)


def test_normals_outward_and_tangent():
    G = oracle_grid(3)
    P = G.points
    for k in range(5):
        assert np.all(np.sum(G.edge_n[:, k] * P, axis=1) < 0)
        assert np.allclose(np.linalg.norm(G.edge_n[:, k], axis=1), 1.0)
        # normal is perpendicular to both corners of the arc
        C = G.corners[G.ring_face[:, k]]
        assert np.max(np.abs(np.sum(G.edge_n[:, k] * C, axis=1))) < 1e-15


def test_spring_dynamics_pentagons_fixed_and_converges():
    pts, faces = og.icosahedron()
    for _ in range(3):
        pts, faces = og.bisect(pts, faces)
    nbr, ring_face, nn = og.neighbour_rings(len(pts), faces)
    P, it, conv = og.spring_dynamics(pts, nbr, nn, 3)
    assert conv and it > 10
    pent = nn == 5
    assert np.array_equal(P[pent], pts[pent])
    assert np.max(np.linalg.norm(P - pts, axis=1)) > 1e-4     # the others moved


def test_spring_natural_length():
    """Eq. dbar at beta = 1.15."""
    assert og.natural_spring_length(4, 1.15) == pytest.approx(1.15 * 2 * np.pi / 80.0, rel=1e-15)


def test_icosahedral_rotation_symmetry():
    """The construction treats the five longitudes alike, so a 72 deg rotation
    about z maps the modified grid onto itself."""
    G = oracle_grid(3)
    a = 2 * np.pi / 5
    R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Q = G.points @ R.T
    from scipy.spatial import cKDTree
    d, _ = cKDTree(G.points).query(Q)
    assert d.max() < 1e-12


def test_centroid_of_symmetric_polygons():
    for n in (3, 5, 6):
        lat = 1.3
        ang = 2 * np.pi * np.arange(n) / n + 0.3
        v = np.stack([np.cos(lat) * np.cos(ang), np.cos(lat) * np.sin(ang), np.full(n, np.sin(lat))], 1)
        c = og.spherical_centroid(v)
        assert np.allclose(c, [0, 0, 1], atol=1e-15)


def test_triangle_area_octant():
    """One octant of the sphere is the triangle (x, y, z) of area pi/2."""
    e = np.eye(3)
    assert og.spherical_triangle_area(e[0], e[1], e[2]) == pytest.approx(np.pi / 2, rel=1e-15)


def test_interpolation_weights_partition():
    """Eq. int_grid weights are positive and sum to one (corners inside)."""
    G = oracle_grid(3)
    assert np.all(G.tri_w > 0)
    assert np.allclose(G.tri_w.sum(1), 1.0, atol=1e-15)


def test_modified_grid_moves_points_to_centroids():
    G = oracle_grid(3)
    for m in (5, 6):
        sel = G.nn == m
        c = og.spherical_centroid(G.corners[G.ring_face[sel, :m]])
        assert np.max(np.abs(c - G.points[sel])) < 1e-15
