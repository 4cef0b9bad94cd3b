"""Pins of the brute-force collision detection references (oracle/detect.py,
Algorithm 1 step 4.1) against hand-solved cases, a library nearest-neighbour
search, a library quadratic program and dense sampling."""
import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial import cKDTree

import oracle
from oracle import detect
import scenes


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- spheres
def test_sphere_hand_cases():
    x = np.array([[0.3, 0.0, 0.0], [0.0, 0.0, 0.5], [2.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.6, 0.0]])
    sph = np.array([[0.0, 0.0, 0.0, 1.0], [0.0, 0.0, 1.2, 1.0]])
    nodes, w, t, c, idx = detect.sphere_springs(np.arange(5), x, sph, 7.0)
    # node 2 is outside both, node 3 sits at the first centre (no direction)
    assert list(idx) == [0, 1, 4]
    np.testing.assert_allclose(t[0], [1.0, 0.0, 0.0], atol=1e-15)
    # node 1: depth 0.5 in sphere 0, 0.3 in sphere 1 -> the deeper one
    np.testing.assert_allclose(t[1], [0.0, 0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(t[2], [0.0, 1.0, 0.0], atol=1e-15)
    assert np.all(c == 7.0) and np.all(nodes[:, 0] == [0, 1, 4]) and np.all(w[:, 0] == 1.0)
    # equal depths: the first sphere wins
    two = np.array([[0.0, 0.0, -1.0, 1.5], [0.0, 0.0, 1.0, 1.5]])
    _, _, t2, _, _ = detect.sphere_springs(np.array([0]), np.zeros((1, 3)), two, 1.0)
    np.testing.assert_allclose(t2[0], [0.0, 0.0, 0.5], atol=1e-15)


def test_sphere_target_is_nearest_surface_point():
    rng = _rng(1)
    sph = np.array([[0.0, 0.0, 0.0, 2.0], [1.5, 0.0, 0.0, 1.0]])
    x = rng.uniform(-2.5, 2.5, size=(300, 3))
    nodes, w, t, c, idx = detect.sphere_springs(np.arange(300), x, sph, 1.0)
    assert len(idx) > 50
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    for j, i in enumerate(idx):
        p = x[i]
        depths = sph[:, 3] - np.linalg.norm(p - sph[:, :3], axis=1)
        q = int(np.argmax(depths))
        assert depths[q] > 0
        surf = sph[q, :3] + sph[q, 3] * u
        dmin = np.linalg.norm(surf - p, axis=1).min()
        d = np.linalg.norm(t[j] - p)
        assert d <= dmin + 1e-12 and dmin - d < 0.05
        assert abs(np.linalg.norm(t[j] - sph[q, :3]) - sph[q, 3]) < 1e-12


# ---------------------------------------------------------------- node pairs
def test_nearest_pair_matches_kdtree():
    rng = _rng(2)
    x = rng.uniform(0, 10, size=(400, 3))
    side_a, side_b = np.arange(0, 150), np.arange(150, 400)
    gap = 1.2
    nodes, w, t, c, idx = detect.nearest_pair_springs(side_a, side_b, x, gap, 3.0)
    d, j = cKDTree(x[side_b]).query(x[side_a])
    act = np.nonzero(d < gap)[0]
    assert list(idx) == list(act)
    assert np.array_equal(nodes[:, 0], side_a[act]) and np.array_equal(nodes[:, 4], side_b[j[act]])
    assert np.all(w[:, 0] == 1.0) and np.all(w[:, 4] == -1.0)
    dv = x[side_a[act]] - x[side_b[j[act]]]
    np.testing.assert_allclose(t, gap * dv / np.linalg.norm(dv, axis=1, keepdims=True), atol=1e-14)


def test_nearest_pair_tie_and_threshold():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 5.0, 0.0]])
    nodes, w, t, c, idx = detect.nearest_pair_springs(np.array([0]), np.array([1, 2]), x, 1.5, 1.0)
    assert nodes[0, 4] == 1                      # equidistant: the first side-B node
    np.testing.assert_allclose(t[0], [-1.5, 0.0, 0.0])
    _, _, _, _, idx = detect.nearest_pair_springs(np.array([3]), np.array([1, 2]), x, 1.5, 1.0)
    assert len(idx) == 0


# ---------------------------------------------------------------- triangles
TRI = (np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))


@pytest.mark.parametrize("p,d2,w", [
    ((0.2, 0.2, 1.0), 1.0, (0.6, 0.2, 0.2)),      # above the interior
    ((-1.0, -1.0, 0.0), 2.0, (1.0, 0.0, 0.0)),    # vertex a region
    ((0.5, -1.0, 0.0), 1.0, (0.5, 0.5, 0.0)),     # edge ab region
    ((1.0, 1.0, 0.0), 0.5, (0.0, 0.5, 0.5)),      # edge bc region
    ((-2.0, 0.5, 3.0), 13.0, (0.5, 0.0, 0.5)),    # edge ca region, off the plane
    ((3.0, -1.0, 0.0), 5.0, (0.0, 1.0, 0.0)),     # vertex b region
])
def test_closest_point_hand_cases(p, d2, w):
    got_d2, got_w, got_q = detect.closest_point_on_triangle(p, *[tuple(v) for v in TRI])
    assert abs(got_d2 - d2) < 1e-14
    np.testing.assert_allclose(got_w, w, atol=1e-15)
    np.testing.assert_allclose(got_q, sum(wi * v for wi, v in zip(w, TRI)), atol=1e-15)


def test_closest_point_against_qp_and_sampling():
    rng = _rng(3)
    s = np.linspace(0, 1, 81)
    S, T = np.meshgrid(s, s)
    keep = S + T <= 1.0
    S, T = S[keep], T[keep]
    for _ in range(60):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 1.5
        d2, wt, _ = detect.closest_point_on_triangle(tuple(p), tuple(a), tuple(b), tuple(c))
        assert min(wt) >= -1e-15 and abs(sum(wt) - 1.0) < 1e-12
        q = wt[0] * a + wt[1] * b + wt[2] * c
        assert abs(np.sum((p - q) ** 2) - d2) < 1e-10
        pts = a[None] + S[:, None] * (b - a)[None] + T[:, None] * (c - a)[None]
        assert d2 <= np.sum((pts - p) ** 2, axis=1).min() + 1e-12
        # the same problem as a library QP over barycentric (s, t)
        f = lambda z: np.sum((a + z[0] * (b - a) + z[1] * (c - a) - p) ** 2)
        cons = [{"type": "ineq", "fun": lambda z: z[0]}, {"type": "ineq", "fun": lambda z: z[1]},
                {"type": "ineq", "fun": lambda z: 1.0 - z[0] - z[1]}]
        r = minimize(f, x0=np.array([1 / 3, 1 / 3]), constraints=cons, method="SLSQP",
                     options={"ftol": 1e-15, "maxiter": 200})
        assert abs(r.fun - d2) < 1e-8 * max(1.0, d2)


def test_point_triangle_springs_hand_cases():
    # one triangle in the plane z = 0 wound counter-clockwise (normal +z)
    X = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 2.0, 0.0],
                  [0.5, 0.5, 2.0], [0.5, 0.5, 2.0], [0.5, 0.5, 2.0], [0.1, 0.1, 0.05]])
    tris = np.array([[0, 1, 2]])
    x = X.copy()
    x[3] = [0.5, 0.5, 0.3]      # in front, within the gap
    x[4] = [0.5, 0.5, -0.2]     # behind (penetrating), within the gap
    x[5] = [0.5, 0.5, 1.0]      # too far
    x[6] = [0.1, 0.1, 0.05]     # near, but already near at rest: excluded
    gap = 0.5
    nodes, w, t, c, idx, which = detect.point_triangle_springs(np.array([3, 4, 5, 6]), tris, x, X, gap, 0.5, 9.0)
    assert list(idx) == [0, 1] and list(which) == [0, 0]
    for j in range(2):
        np.testing.assert_allclose(t[j], [0.0, 0.0, gap], atol=1e-15)
        np.testing.assert_allclose(-w[j, 4:7], [0.5, 0.25, 0.25], atol=1e-15)
        assert list(nodes[j, 4:7]) == [0, 1, 2]
    # a node beyond the edge x = 0, in front: pushed along q -> node, not along n
    X2 = np.vstack([X[:3], [[-0.3, 0.5, 3.0]]])
    x2 = X2.copy()
    x2[3] = [-0.3, 0.5, 0.4]
    _, w2, t2, _, idx2, _ = detect.point_triangle_springs(np.array([3]), tris, x2, X2, 0.6, 0.5, 1.0)
    assert list(idx2) == [0]
    np.testing.assert_allclose(t2[0], [-0.36, 0.0, 0.48], atol=1e-15)
    np.testing.assert_allclose(-w2[0, 4:7], [0.75, 0.0, 0.25], atol=1e-15)
    # the spring's rest point is the node a distance gap in front of q
    con = scenes.Contacts(nodes[:1], w[:1], t[:1], c[:1])
    xr = x.copy()
    xr[3] = [0.5, 0.5, gap]
    f = oracle.contact_forces(con, xr)
    assert np.abs(f).max() < 1e-12
    f = oracle.contact_forces(con, x)
    np.testing.assert_allclose(f[3], [0.0, 0.0, 9.0 * (gap - 0.3)], atol=1e-12)
    np.testing.assert_allclose(f[:3].sum(axis=0), -f[3], atol=1e-12)


def test_point_triangle_nearest_and_tie():
    # two triangles sharing an edge in one plane: a node above the shared edge
    # is equidistant (first index), a node over the second one picks it
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0.5, 0.5, 3], [0.8, 0.9, 3]], float)
    tris = np.array([[0, 1, 2], [1, 3, 2]])
    x = X.copy()
    x[4] = [0.5, 0.5, 0.2]
    x[5] = [0.8, 0.9, 0.1]
    _, w, t, _, idx, which = detect.point_triangle_springs(np.array([4, 5]), tris, x, X, 0.4, 1.0, 1.0)
    assert list(which) == [0, 1]
    np.testing.assert_allclose(-w[0, 4:7], [0.0, 0.5, 0.5], atol=1e-15)


def test_outward_faces_of_a_box():
    X, tets, _ = scenes.grid_mesh(2, 1, 1)
    faces = scenes.boundary_faces_outward(X, tets)
    assert len(faces) == 2 * (2 * 2 + 2 * 1 + 2 * 2)   # two triangles per unit square of the surface
    a, b, c = (X[faces[:, i]] for i in range(3))
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    assert np.all(np.sum(n * (cen - X.mean(axis=0)), axis=1) > 0)
    # the face normals integrate to zero over a closed surface
    np.testing.assert_allclose(n.sum(axis=0), 0.0, atol=1e-12)
