"""Nested Schur refactorisation of the FP64 form (pd_set_contact_nodes): the
same solve H u = g as the plain form, checked against the oracle."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_util import need_gpu, rng, contact_tuple, region_callback, oracle_callback, assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _solver(pd, s, **kw):
    return pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt, **kw)


def _oracle_H(s, c):
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    S0 = oracle.schur_complement(o.K, o.part.x1, o.part.region)
    H = S0.copy()
    if c.k:
        H += oracle.contact_matrix(c, len(s.X)).toarray()[np.ix_(s.region, s.region)]
    return H


@pytest.mark.parametrize("which", ["proxies", "one", "all"])
def test_nested_solve_matches_oracle_and_plain(pd, which):
    s = scenes.small_elbow(h=1.5)
    step = 56
    c = s.contacts(step, s.X)
    if which == "proxies":
        nodes = s.proxies
    elif which == "one":
        nodes = np.unique(c.nodes[c.nodes >= 0])[:1]
        keep = np.all(np.isin(c.nodes, np.r_[nodes, -1]), axis=1)
        c = scenes.Contacts(c.nodes[keep], c.w[keep], c.target[keep], c.stiffness[keep])
    else:
        nodes = s.region
    assert c.k > 0
    H = _oracle_H(s, c)
    g = rng(81).normal(size=(s.m, 3)) * 1e3
    plain = _solver(pd, s)
    plain.set_contacts(*contact_tuple(c))
    up = plain.schur_solve(g)
    sol = _solver(pd, s)
    sol.set_contact_nodes(nodes)
    sol.set_contacts(*contact_tuple(c))
    u = sol.schur_solve(g)
    res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
    assert res <= TOL, res
    assert np.linalg.norm(u - up) / np.linalg.norm(up) <= 1e-12
    # springs changed: only the trailing block is refactored again
    c2 = scenes.Contacts(c.nodes, c.w, c.target, 3.0 * c.stiffness)
    sol.set_contacts(*contact_tuple(c2))
    u2 = sol.schur_solve(g)
    H2 = _oracle_H(s, c2)
    assert np.linalg.norm(g - H2 @ u2) / np.linalg.norm(g) <= TOL


def test_nested_outer_iterations_match_oracle(pd):
    s = scenes.small_elbow(h=1.5, inner_iters=2)
    step = 56
    x0 = s.X.copy()
    sol = _solver(pd, s, inner_iters=2)
    sol.set_contact_nodes(s.proxies)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(step))
    sol.step(2, region_callback(s, step, x0))
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(2, 2, oracle_callback(s, step), s.dirichlet_positions(step))
    assert_parity(sol.positions(), xo, x0, TOL)


def test_nested_with_device_pair_detector(pd):
    s = scenes.small_elbow(h=1.5)
    x0 = s.X.copy()
    side_a, side_b = s.info["pair_sides"]
    sol = _solver(pd, s, inner_iters=2)
    sol.set_contact_nodes(s.proxies)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(50))
    sol.set_detector_pairs(side_a, side_b, 6.0, s.stiffness)
    sol.step(2)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(2, 2, lambda x: s.info["self_pairs"](x, gap=6.0), s.dirichlet_positions(50))
    assert_parity(sol.positions(), xo, x0, TOL)


def test_nested_rejects_springs_on_other_nodes(pd):
    s = scenes.small_elbow(h=1.5)
    sol = _solver(pd, s)
    sol.set_contact_nodes(s.proxies)
    inner = np.setdiff1d(s.region, s.proxies)[:1]
    nodes = np.full((1, 4), -1, np.int32)
    nodes[0, 0] = inner[0]
    w = np.zeros((1, 4)); w[0, 0] = 1.0
    with pytest.raises(RuntimeError):
        sol.set_contacts(nodes, w, s.X[inner], np.array([1e6]))
    with pytest.raises(RuntimeError):
        sol.set_detector_spheres(inner, np.array([[0.0, 0.0, 0.0, 1.0]]), 1e6)
    # turning it off accepts them again
    sol.set_contact_nodes(None)
    sol.set_contacts(nodes, w, s.X[inner], np.array([1e6]))


@pytest.mark.parametrize("prec", ["FP32_IR", "TF32_IR", "BF16_IR"])
def test_nested_mixed_forms(pd, prec):
    s = scenes.small_elbow(h=1.5)
    step = 56
    c = s.contacts(step, s.X)
    H = _oracle_H(s, c)
    g = rng(83).normal(size=(s.m, 3)) * 1e3
    sol = _solver(pd, s, max_refine=500)
    sol.set_contact_nodes(s.proxies)
    sol.set_precision(getattr(pd, prec))
    for rep in range(2):   # the second solve starts from the saved trailing block
        sol.set_contacts(*contact_tuple(c))
        u = sol.schur_solve(g)
        res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
        assert res <= TOL, (prec, rep, res)
    # one outer iteration vs the oracle
    x0 = s.X.copy()
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(step))
    sol.step(1, region_callback(s, step, x0))
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(1, 1, oracle_callback(s, step), s.dirichlet_positions(step))
    assert_parity(sol.positions(), xo, x0, 1e-8)
