"""Collision detection on the device (Algorithm 1, step 4.1) vs the oracle
with the same detection done on the host at every inner iteration, by the
brute-force references of oracle/detect.py."""
import numpy as np
import pytest

import oracle
from oracle import detect
import scenes
from gpu_util import need_gpu, rng, assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _solver(pd, s, **kw):
    return pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt, **kw)


def _oracle(s):
    return oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)


def _spheres_fn(proxies, spheres, stiffness):
    return lambda x: scenes.Contacts(*detect.sphere_springs(proxies, x, spheres, stiffness)[:4])


def _pairs_fn(side_a, side_b, gap, stiffness):
    return lambda x: scenes.Contacts(*detect.nearest_pair_springs(side_a, side_b, x, gap, stiffness)[:4])


def test_sphere_detector_trajectory_matches_oracle(pd):
    # 3 backward-Euler steps x 10 outer x 2 inner iterations, the descending
    # sphere re-detected against the current x_2 at every inner iteration
    s = scenes.config1(pre_indent=0.7)
    s_inner = 2
    sol = _solver(pd, s, inner_iters=s_inner)
    o = _oracle(s)
    centre = s.info["sphere_centre"]
    active = 0
    for st in range(3):
        sph = np.r_[centre(st), 3.0][None, :]
        fn = _spheres_fn(s.proxies, sph, s.stiffness)
        sol.set_dirichlet(s.dirichlet_positions(st))
        sol.set_detector_spheres(s.proxies, sph, s.stiffness)
        sol.step(s.outer_iters)
        o.step(s.outer_iters, s_inner, fn, s.dirichlet_positions(st))
        active = max(active, fn(o.x).k)
    xg, vg = sol.get_state()
    assert active > 0
    assert_parity(xg, o.x, s.X, 1e-8, "positions")
    assert_parity(vg, o.v, np.zeros_like(o.v), 1e-8, "velocities")
    assert sol.stats()["contacts"] == len(s.proxies)


def test_sphere_detector_equals_host_callback(pd):
    # same step with detection on the device and through the host callback
    s = scenes.config1(pre_indent=0.8, nx=6, ny=6, nz=12)
    x0 = s.X.copy()
    free = np.setdiff1d(np.arange(s.n), s.dirichlet)
    x0[free] += 0.03 * rng(41).normal(size=(len(free), 3))
    c = s.info["sphere_centre"](0)
    spheres = np.array([[*c, 3.0], [c[0] + 40.0, c[1], c[2], 1.0]])   # second sphere far away
    a = _solver(pd, s, inner_iters=3)
    a.set_state(x0)
    a.set_detector_spheres(s.proxies, spheres, s.stiffness)
    a.step(2)
    b = _solver(pd, s, inner_iters=3)
    b.set_state(x0)

    fn = _spheres_fn(s.proxies, spheres, s.stiffness)

    def cb(x2):
        x = x0.copy()
        x[s.region] = x2
        cc = fn(x)
        return (cc.nodes, cc.w, cc.target, cc.stiffness)

    b.step(2, cb)
    xa, xb = a.positions(), b.positions()
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xb - x0) <= TOL


def test_pair_detector_matches_oracle(pd):
    # two-sided self-collision springs re-detected on the device
    s = scenes.small_elbow(h=1.5)
    x0 = s.X.copy()
    side_a, side_b = s.info["pair_sides"]
    fn = _pairs_fn(side_a, side_b, 6.0, s.stiffness)
    assert fn(x0).k > 5
    sol = _solver(pd, s, inner_iters=2)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(50))
    sol.set_detector_pairs(side_a, side_b, 6.0, s.stiffness)
    sol.step(2)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(2, 2, fn, s.dirichlet_positions(50))
    assert_parity(sol.positions(), xo, x0, TOL)


def test_detector_errors_and_clear(pd):
    s = scenes.config1(nx=3, ny=3, nz=5)
    sol = _solver(pd, s)
    x0 = sol.positions()
    outside = np.setdiff1d(np.arange(s.n), s.region)[:1]
    with pytest.raises(RuntimeError):
        sol.set_detector_spheres(outside, np.array([[0, 0, 0, 1.0]]), 1e6)
    with pytest.raises(RuntimeError):
        sol.set_detector_pairs(s.proxies, s.proxies, -1.0, 1e6)
    # an empty side B: every slot inactive, same as no springs
    sol.set_detector_pairs(s.proxies, np.zeros(0, np.int32), 1.0, 1e6)
    sol.step(2)
    x_det = sol.positions()
    sol.set_state(x0)
    sol.clear_detector()
    sol.step(2)
    assert np.array_equal(x_det, sol.positions())
    # a sphere that touches nothing
    sol.set_state(x0)
    sol.set_detector_spheres(s.proxies, np.array([[100.0, 0, 0, 1.0]]), 1e6)
    sol.step(2)
    assert np.array_equal(x_det, sol.positions())


def _closed_elbow(h=1.5, frac=0.08, angle=40.0, band=8.0):
    """Small elbow in the closed-joint pose (no element inverted; side-A
    nodes within the gap of side-B triangles) and the matching caps."""
    s = scenes.small_elbow(h=h, region_fraction=frac)
    x0, step = scenes.closed_pose(s, angle, band)
    return s, x0, s.dirichlet_positions(step)


def _tri_fn(s):
    pa, ta, pb, tb = s.info["tri_sides"]
    gap, rmin = s.info["tri_gap"], s.info["tri_rest_min"]

    def fn(x):
        A = detect.point_triangle_springs(pa, tb, x, s.X, gap, rmin, s.stiffness)
        B = detect.point_triangle_springs(pb, ta, x, s.X, gap, rmin, s.stiffness)
        return scenes.Contacts(*(np.concatenate([A[i], B[i]]) for i in range(4)))

    return fn


def _set_tri(sol, s):
    pa, ta, pb, tb = s.info["tri_sides"]
    sol.set_detector_triangles(pa, ta, pb, tb, s.info["tri_gap"], s.info["tri_rest_min"], s.stiffness)


def _compare_springs(sol, s, x):
    nodes, w, t, c = sol.contacts()
    pa, ta, pb, tb = s.info["tri_sides"]
    assert len(c) == len(pa) + len(pb)
    ref = _tri_fn(s)(x)
    act = c > 0
    assert act.sum() == ref.k
    np.testing.assert_array_equal(nodes[act], ref.nodes)
    np.testing.assert_array_equal(w[act], ref.w)
    np.testing.assert_array_equal(t[act], ref.target)
    np.testing.assert_array_equal(c[act], ref.stiffness)
    assert np.all(nodes[~act] == -1) and np.all(w[~act] == 0.0)
    return ref.k


def test_triangle_detector_springs_equal_oracle(pd):
    # the detected springs themselves -- which nodes are active, which
    # triangle and closest point (decisions bit for bit), weights, targets --
    # on the closed pose and again on the state one solver step later (the
    # same positions go to both sides)
    s, x0, dpos = _closed_elbow()
    sol = _solver(pd, s)
    sol.set_state(x0)
    _set_tri(sol, s)
    sol.detect()
    assert _compare_springs(sol, s, x0) >= 20
    sol.set_dirichlet(dpos)
    sol.step(1)
    x1 = sol.positions()
    sol.detect()
    assert _compare_springs(sol, s, x1) >= 5


def test_triangle_detector_steps_match_oracle_from_the_same_state(pd):
    # three outer iterations from the closed pose, the springs re-detected on
    # the device; each compared with the oracle's iteration from the same
    # state (a node equidistant from two surfaces makes the nearest-triangle
    # choice discontinuous, so two runs apart by rounding may pick
    # differently later; the same state gives the same choice)
    s, x0, dpos = _closed_elbow()
    fn = _tri_fn(s)
    assert fn(x0).k >= 20
    sol = _solver(pd, s)
    sol.set_state(x0)
    sol.set_dirichlet(dpos)
    _set_tri(sol, s)
    x = x0.copy()
    for it in range(3):
        sol.step(1)
        xg = sol.positions()
        o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
        o.x = x.copy()
        xo = o.step(1, 1, fn, dpos)
        scale = np.abs(xo - x).max()
        err_node = np.abs(xg - xo).max() / scale
        err = np.linalg.norm(xg - xo) / np.linalg.norm(xo - x)
        assert err_node <= TOL and err <= TOL, (it, err_node, err)
        x = xg


def test_triangle_detector_errors(pd):
    s, x0, dpos = _closed_elbow(h=2.0, frac=0.05)
    sol = _solver(pd, s)
    pa, ta, pb, tb = s.info["tri_sides"]
    outside = np.setdiff1d(np.arange(s.n), s.region)[:1]
    with pytest.raises(RuntimeError):
        sol.set_detector_triangles(outside, ta, pb, tb, 1.0, 1.0, 1e6)
    bad = ta.copy()
    bad[0, 1] = outside[0]
    with pytest.raises(RuntimeError):
        sol.set_detector_triangles(pa, bad, pb, tb, 1.0, 1.0, 1e6)
    with pytest.raises(RuntimeError):
        sol.set_detector_triangles(pa, ta, pb, tb, 0.0, 1.0, 1e6)
    with pytest.raises(RuntimeError):
        sol.set_detector_triangles(pa, ta, pb, tb, 1.0, -1.0, 1e6)
    with pytest.raises(RuntimeError):
        sol.detect()                      # no detector set
    # at rest nothing is within the gap: every slot empty
    sol.set_detector_triangles(pa, ta, pb, tb, s.info["tri_gap"], s.info["tri_rest_min"], 1e6)
    sol.detect()
    _, _, _, c = sol.contacts()
    assert len(c) == len(pa) + len(pb) and np.all(c == 0.0)
