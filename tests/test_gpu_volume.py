"""The PD volume term kappa ||F - T||^2 (the lambda term of Eq. 1 in PD
form, det T bounded) on the device vs the FP64 oracle: local-step forces
(inverted elements included, alone and together with the bi-phasic term),
one outer iteration, a backward-Euler trajectory, the elbow bend and the
mixed-precision forms."""
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


def _solver(pd, s, kappa, lo, hi, **kw):
    return pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt,
                     kappa=kappa, det_min=lo, det_max=hi, **kw)


def _oracle(s, kappa, lo, hi, **kw):
    return oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt,
                               kappa=kappa, det_min=lo, det_max=hi, **kw)


def _well_conditioned_t(F, T):
    # T = U diag(tau) V^T on the principal branch tau_i = (s_i + r_i) / 2;
    # dtau / ds grows like 1 / r_i, so within 5% of the branch end
    # (min r_i < 0.05 max |s_i|) rounding-level differences in s become
    # ~sqrt(eps) differences in T: such elements are left out
    from oracle import pd_oracle
    U, sv, Vt = pd_oracle.signed_svd(F)
    tau = np.diagonal(np.swapaxes(U, 1, 2) @ T @ np.swapaxes(Vt, 1, 2), axis1=1, axis2=2)
    r = np.abs(2.0 * tau - sv)
    moved = np.abs(T - F).max(axis=(1, 2)) > 0
    return ~moved | (r.min(axis=1) >= 0.05 * np.abs(sv).max(axis=1))


def _unique_r(F):
    # R (and so S's eigenvectors) is unique where the two smallest signed
    # singular values are apart
    U, S, Vt = np.linalg.svd(F)
    d = np.sign(np.linalg.det(U @ Vt))
    return (S[:, 1] + d * S[:, 2]) / S[:, 0] > 1e-3


@pytest.mark.parametrize("with_strain_limit", [False, True])
def test_local_step_forces_match_oracle(pd, with_strain_limit):
    s = scenes.config1(nx=5, ny=5, nz=8)
    lo, hi, kappa = 0.95, 1.05, 6 * s.mu
    mp, slo, shi = (4 * s.mu, 0.9, 1.1) if with_strain_limit else (0.0, 0.0, np.inf)
    x = s.X * np.array([1.15, 0.9, 1.0]) + 0.08 * rng(61).normal(size=s.X.shape)
    for e in rng(62).choice(s.E, 6, replace=False):   # a few inverted elements
        a, b = s.tets[e, 0], s.tets[e, 1]
        x[[a, b]] = x[[b, a]]
    sol = _solver(pd, s, kappa, lo, hi, mu_prime=mp, sigma_min=slo, sigma_max=shi)
    R, f = sol.local_step(x)
    o = _oracle(s, kappa, lo, hi, mu_prime=mp, sigma_min=slo, sigma_max=shi)
    all_e = np.arange(s.E)
    F = oracle.deformation_gradients(x, o.tets, o.Dm_inv)
    det = np.linalg.det(F)
    assert (det < lo).any() and (det > hi).any() and (det < 0).any()
    Ro = o.rotations(x, all_e)
    To = o.volume_targets(x, all_e)
    keep = _unique_r(F) & _well_conditioned_t(F, To)
    fo = (oracle.elastic_forces(x, Ro, o.tets, o.Dm_inv, o.vol, o.mu)
          + oracle.elastic_forces(x, To, o.tets, o.Dm_inv, o.vol, kappa))
    if with_strain_limit:
        fo += oracle.elastic_forces(x, o.projections(x, all_e), o.tets, o.Dm_inv, o.vol, mp)
    assert keep.mean() > 0.97
    assert np.abs(R[keep] - Ro[keep]).max() <= 1e-12
    bad = np.zeros(s.n, bool)
    bad[s.tets[~keep].ravel()] = True
    assert (~bad).sum() > 0.9 * s.n
    assert np.abs(f[~bad] - fo[~bad]).max() <= TOL * np.abs(fo).max()


def test_rest_state_has_no_volume_force(pd):
    # at rest det F = 1 up to rounding, on either side of the bound: T = F up
    # to rounding (the projection's Newton iteration must not stop at the
    # branch end, where its slope is unbounded)
    s = scenes.config1(nx=5, ny=5, nz=8)
    sol = _solver(pd, s, 1.5 * s.lam, 1.0, 1.0)
    _, f = sol.local_step(s.X.copy())
    assert np.abs(f).max() <= 1e-8, np.abs(f).max()


@pytest.mark.parametrize("inner", [1, 3])
def test_one_outer_iteration_matches_oracle(pd, inner):
    # the lambda term of configuration 1 (lambda = 4e4) in PD form:
    # kappa = 3 lambda / 2, det T = 1
    s = scenes.config1(pre_indent=0.7, nx=6, ny=6, nz=12)
    kappa = 1.5 * s.lam
    x0 = s.X.copy()
    free = np.setdiff1d(np.arange(s.n), s.dirichlet)
    x0[free] += 0.03 * rng(63).normal(size=(len(free), 3))
    sol = _solver(pd, s, kappa, 1.0, 1.0, inner_iters=inner)
    sol.set_state(x0)
    sol.step(1, region_callback(s, 0, x0))
    o = _oracle(s, kappa, 1.0, 1.0)
    o.x = x0.copy()
    xo = o.step(1, inner, oracle_callback(s, 0), s.dirichlet_positions(0))
    assert_parity(sol.positions(), xo, x0, TOL)


def test_trajectory_matches_oracle_and_keeps_volume(pd):
    # 3 backward-Euler steps x 10 outer iterations, the sphere pressing in
    s = scenes.config1(pre_indent=0.9, nx=5, ny=5, nz=10)
    kappa = 1.5 * s.lam
    sol = _solver(pd, s, kappa, 1.0, 1.0)
    o = _oracle(s, kappa, 1.0, 1.0)
    for st in range(3):
        xg_prev = sol.positions()
        sol.set_dirichlet(s.dirichlet_positions(st))
        sol.step(s.outer_iters, region_callback(s, st, xg_prev))
        o.step(s.outer_iters, 1, oracle_callback(s, st), s.dirichlet_positions(st))
    assert_parity(sol.positions(), o.x, s.X, 1e-8)
    # the same run without the term changes volume more
    p = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt)
    for st in range(3):
        xg_prev = p.positions()
        p.set_dirichlet(s.dirichlet_positions(st))
        p.step(s.outer_iters, region_callback(s, st, xg_prev))
    dv = [np.abs(np.linalg.det(oracle.deformation_gradients(xx, o.tets, o.Dm_inv)) - 1.0).mean()
          for xx in (sol.positions(), p.positions())]
    assert dv[0] < dv[1], dv


def test_elbow_bend_matches_oracle(pd):
    s = scenes.small_elbow(inner_iters=2)
    kappa, lo, hi = 10 * s.mu, 0.97, 1.03
    step = 52
    x0 = s.X.copy()
    sol = _solver(pd, s, kappa, lo, hi, inner_iters=2)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(step))
    sol.step(3, region_callback(s, step, x0))
    o = _oracle(s, kappa, lo, hi)
    o.x = x0.copy()
    xo = o.step(3, 2, oracle_callback(s, step), s.dirichlet_positions(step))
    assert_parity(sol.positions(), xo, x0, TOL)


@pytest.mark.parametrize("prec", ["FP32_IR", "BF16_IR"])
def test_mixed_forms_with_volume_term_match_fp64(pd, prec):
    s = scenes.config1(pre_indent=0.7, nx=6, ny=6, nz=12)
    kappa = 1.5 * s.lam
    x0 = s.X.copy()
    out = []
    for p in (pd.FP64, getattr(pd, prec)):
        sol = _solver(pd, s, kappa, 1.0, 1.0, inner_iters=2, precision=p, max_refine=200)
        sol.set_state(x0)
        sol.step(4, region_callback(s, 0, x0))
        out.append(sol.positions())
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0] - x0) <= 1e-8


def test_invalid_volume_arguments(pd):
    s = scenes.config1(nx=3, ny=3, nz=4)
    for kappa, lo, hi in ((s.mu, 1.2, 0.8), (-1.0, 1.0, 1.0), (s.mu, 0.0, 1.0), (s.mu, np.nan, 1.0),
                          (np.inf, 1.0, 1.0)):
        with pytest.raises(RuntimeError):
            _solver(pd, s, kappa, lo, hi)
