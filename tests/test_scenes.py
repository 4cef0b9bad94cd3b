"""The seeded scene generators: sizes, orientation and conformity."""
import numpy as np
import pytest

import scenes
from scenes.mesh import boundary_faces


def test_config1_sizes():
    s = scenes.config1()
    assert (s.n, s.E) == (11 * 11 * 41, 20000)
    assert len(s.dirichlet) == 121 and s.m == 242 and len(s.proxies) == 121
    assert not np.intersect1d(s.dirichlet, s.region).size


def test_grid_is_conforming_and_positive():
    X, tets, _ = scenes.grid_mesh(3, 4, 5)
    a, b, c, d = (X[tets[:, i]] for i in range(4))
    det = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    assert np.all(det > 0)
    # a conforming box mesh has exactly 2 boundary triangles per boundary square
    assert len(boundary_faces(tets)) == 2 * 2 * (3 * 4 + 4 * 5 + 3 * 5)


def test_seeded_jitter_is_reproducible():
    a, b = scenes.config1(seed=3), scenes.config1(seed=3)
    np.testing.assert_array_equal(a.X, b.X)
    assert not np.array_equal(a.X, scenes.config1(seed=4).X)


def test_small_elbow_region():
    s = scenes.small_elbow()
    inr = np.zeros(s.n, bool)
    inr[s.region] = True
    assert s.m == int(np.ceil(0.05 * s.n))
    assert not np.any(inr[s.dirichlet])
    assert np.all(inr[s.proxies])


def test_sphere_contacts_project_to_surface():
    s = scenes.config1(pre_indent=0.5)
    c = s.contacts(0, s.X)
    assert c.k > 1
    ctr = s.info["sphere_centre"](0)
    np.testing.assert_allclose(np.linalg.norm(c.target - ctr, axis=1), 3.0, atol=1e-12)
