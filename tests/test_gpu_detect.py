"""Collision detection on the device (Algorithm 1, step 4.1) vs the oracle
with the same detection done on the host at every inner iteration."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_util import need_gpu, rng

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
        sol.set_dirichlet(s.dirichlet_positions(st))
        sol.set_detector_spheres(s.proxies, np.r_[centre(st), 3.0][None, :], s.stiffness)
        sol.step(s.outer_iters)
        o.step(s.outer_iters, s_inner, lambda x, st=st: s.contacts(st, x), s.dirichlet_positions(st))
        active = max(active, s.contacts(st, o.x).k)
    xg, vg = sol.get_state()
    assert active > 0
    err = np.linalg.norm(xg - o.x) / np.linalg.norm(o.x - s.X)
    assert err <= 1e-8, err
    assert np.linalg.norm(vg - o.v) / np.linalg.norm(o.v) <= 1e-8
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

    def cb(x2):
        x = x0.copy()
        x[s.region] = x2
        cc = scenes.sphere_contacts(s.proxies, x, c, 3.0, s.stiffness)
        return (cc.nodes, cc.w, cc.target, cc.stiffness)

    b.step(2, cb)
    xa, xb = a.positions(), b.positions()
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xb - x0) <= TOL


def test_pair_detector_matches_oracle(pd):
    # two-sided self-collision springs re-detected on the device
    s = scenes.small_elbow(h=1.5)
    x0 = s.X.copy()
    fn = s.info["self_pairs"]
    assert fn(x0, gap=6.0).k > 5
    side_a, side_b = s.info["pair_sides"]
    sol = _solver(pd, s, inner_iters=2)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(50))
    sol.set_detector_pairs(side_a, side_b, 6.0, s.stiffness)
    sol.step(2)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(2, 2, lambda x: fn(x, gap=6.0), s.dirichlet_positions(50))
    err = np.linalg.norm(sol.positions() - xo) / np.linalg.norm(xo - x0)
    assert err <= TOL, err


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
