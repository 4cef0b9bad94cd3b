"""Bi-phasic strain limiting (Section 5) on the device vs the FP64 oracle."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_util import need_gpu, rng, region_callback, oracle_callback, assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _solver(pd, s, mp, lo, hi, **kw):
    return pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt,
                     mu_prime=mp, sigma_min=lo, sigma_max=hi, **kw)


def _oracle(s, mp, lo, hi):
    return oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt,
                               mu_prime=mp, sigma_min=lo, sigma_max=hi)


def test_local_step_forces_match_oracle(pd):
    s = scenes.config1(nx=5, ny=5, nz=8)
    lo, hi, mp = 0.9, 1.1, 6 * s.mu
    x = s.X * np.array([1.15, 0.9, 1.0]) + 0.08 * rng(51).normal(size=s.X.shape)
    # a few inverted elements: swap two vertices' positions of some tets
    for e in rng(52).choice(s.E, 6, replace=False):
        a, b = s.tets[e, 0], s.tets[e, 1]
        x[[a, b]] = x[[b, a]]
    sol = _solver(pd, s, mp, lo, hi)
    R, f = sol.local_step(x)
    o = _oracle(s, mp, lo, hi)
    all_e = np.arange(s.E)
    F = oracle.deformation_gradients(x, o.tets, o.Dm_inv)
    sv = np.linalg.svd(F, compute_uv=False)
    assert (sv > hi).any() and (sv < lo).any() and (np.linalg.det(F) < 0).any()
    # compare only where R is unique (the two smallest signed singular values apart)
    U, S, Vt = np.linalg.svd(F)
    d = np.sign(np.linalg.det(U @ Vt))
    margin = (S[:, 1] + d * S[:, 2]) / S[:, 0]
    keep = margin > 1e-3
    Ro = o.rotations(x, all_e)
    Qo = o.projections(x, all_e)
    fo = (oracle.elastic_forces(x, Ro, o.tets, o.Dm_inv, o.vol, o.mu)
          + oracle.elastic_forces(x, Qo, o.tets, o.Dm_inv, o.vol, o.mu_prime))
    assert keep.mean() > 0.99
    assert np.abs(R[keep] - Ro[keep]).max() <= 1e-12
    # nodes whose every element has a unique R
    bad = np.zeros(s.n, bool)
    bad[s.tets[~keep].ravel()] = True
    assert (~bad).sum() > 0.9 * s.n
    assert np.abs(f[~bad] - fo[~bad]).max() <= TOL * np.abs(fo).max()


@pytest.mark.parametrize("inner", [1, 3])
def test_one_outer_iteration_matches_oracle(pd, inner):
    s = scenes.config1(pre_indent=0.7, nx=6, ny=6, nz=12)
    lo, hi, mp = 0.97, 1.03, 5 * s.mu
    x0 = s.X.copy()
    free = np.setdiff1d(np.arange(s.n), s.dirichlet)
    x0[free] += 0.03 * rng(53).normal(size=(len(free), 3))
    sol = _solver(pd, s, mp, lo, hi, inner_iters=inner)
    sol.set_state(x0)
    sol.step(1, region_callback(s, 0, x0))
    o = _oracle(s, mp, lo, hi)
    o.x = x0.copy()
    xo = o.step(1, inner, oracle_callback(s, 0), s.dirichlet_positions(0))
    assert_parity(sol.positions(), xo, x0, TOL)


def test_trajectory_matches_oracle(pd):
    # 3 backward-Euler steps x 10 outer iterations, the sphere pressing in
    s = scenes.config1(pre_indent=0.9, nx=5, ny=5, nz=10)
    lo, hi, mp = 0.95, 1.05, 8 * s.mu
    sol = _solver(pd, s, mp, lo, hi)
    o = _oracle(s, mp, lo, hi)
    for st in range(3):
        xg_prev = sol.positions()
        sol.set_dirichlet(s.dirichlet_positions(st))
        sol.step(s.outer_iters, region_callback(s, st, xg_prev))
        o.step(s.outer_iters, 1, oracle_callback(s, st), s.dirichlet_positions(st))
    assert_parity(sol.positions(), o.x, s.X, 1e-8)
    F = oracle.deformation_gradients(o.x, o.tets, o.Dm_inv)
    sv = np.linalg.svd(F, compute_uv=False)
    assert (sv > hi).any() or (sv < lo).any()


def test_elbow_bend_matches_oracle_and_limits_strain(pd):
    s = scenes.small_elbow(inner_iters=2)
    lo, hi, mp = 0.9, 1.1, 20 * s.mu
    step = 52
    x0 = s.X.copy()
    sol = _solver(pd, s, mp, lo, hi, inner_iters=2)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(step))
    sol.step(3, region_callback(s, step, x0))
    o = _oracle(s, mp, lo, hi)
    o.x = x0.copy()
    xo = o.step(3, 2, oracle_callback(s, step), s.dirichlet_positions(step))
    assert_parity(sol.positions(), xo, x0, TOL)


def test_mixed_form_with_strain_limit_matches_fp64(pd):
    s = scenes.config1(pre_indent=0.7, nx=6, ny=6, nz=12)
    lo, hi, mp = 0.97, 1.03, 5 * s.mu
    x0 = s.X.copy()
    out = []
    for prec in (pd.FP64, pd.TF32_IR):
        sol = _solver(pd, s, mp, lo, hi, inner_iters=2, precision=prec)
        sol.set_state(x0)
        sol.step(4, region_callback(s, 0, x0))
        out.append(sol.positions())
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0] - x0) <= 1e-8


def test_invalid_strain_limit_arguments(pd):
    s = scenes.config1(nx=3, ny=3, nz=4)
    with pytest.raises(RuntimeError):
        _solver(pd, s, s.mu, 1.2, 0.8)
    with pytest.raises(RuntimeError):
        _solver(pd, s, -1.0, 0.8, 1.2)
    with pytest.raises(RuntimeError):
        _solver(pd, s, s.mu, np.nan, 1.2)
