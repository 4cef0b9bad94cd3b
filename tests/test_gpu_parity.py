"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import scenes
from gpu_util import need_gpu, rng, contact_tuple, region_callback, oracle_callback, parity_errors, assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10      # relative tolerance of the FP64 form


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _solver(pd, s, **kw):
    return pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt, **kw)


def _unique_rotation_margin(F):
    U, S, Vt = np.linalg.svd(F)
    d = np.sign(np.linalg.det(U @ Vt))
    return (S[:, 1] + d * S[:, 2]) / np.maximum(S[:, 0], 1e-300)


def test_local_step_matches_oracle(pd):
    s = scenes.config1()
    x = s.X + 0.12 * rng(1).normal(size=s.X.shape)
    sol = _solver(pd, s)
    R, f = sol.local_step(x)
    Dm_inv, vol = oracle.element_precompute(s.X, s.tets.astype(np.int64))
    F = oracle.deformation_gradients(x, s.tets.astype(np.int64), Dm_inv)
    Ro = oracle.polar_rotations(F)
    assert _unique_rotation_margin(F).min() > 1e-2
    assert np.abs(R - Ro).max() <= TOL
    fo = oracle.elastic_forces(x, Ro, s.tets.astype(np.int64), Dm_inv, vol, s.mu)
    assert np.abs(f - fo).max() <= TOL * np.abs(fo).max()


def test_local_step_inverted_and_degenerate_elements(pd):
    s = scenes.config1(nx=4, ny=4, nz=4)
    x = s.X.copy()
    g = rng(2)
    # invert a handful of tets by pushing interior nodes through their neighbours
    inner = np.nonzero(np.all((s.X > 0.5) & (s.X < 3.5), axis=1))[0]
    pick = g.choice(inner, 6, replace=False)
    x[pick] += g.normal(size=(6, 3)) * 1.5
    x[inner[:2]] = x[inner[2]]            # two coincident nodes: rank-deficient F
    sol = _solver(pd, s)
    R, _ = sol.local_step(x)
    Dm_inv, vol = oracle.element_precompute(s.X, s.tets.astype(np.int64))
    F = oracle.deformation_gradients(x, s.tets.astype(np.int64), Dm_inv)
    Ro = oracle.polar_rotations(F)
    det = np.linalg.det(F)
    assert np.sum(det < 0) > 0
    RtR = np.einsum("eji,ejk->eik", R, R)
    assert np.abs(RtR - np.eye(3)).max() <= 1e-12
    assert np.abs(np.linalg.det(R) - 1.0).max() <= 1e-12
    psi = np.sum((F - R) ** 2, axis=(1, 2))
    psio = np.sum((F - Ro) ** 2, axis=(1, 2))
    # the minimum is unique in value even where the minimiser is not
    assert np.all(psi <= psio + 1e-12 * np.maximum(1.0, psio))
    uniq = _unique_rotation_margin(F) > 1e-3
    assert np.abs(R[uniq] - Ro[uniq]).max() <= 1e-9


def _oracle_H(s, contacts, mass_dt=True):
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    K = o.K if o.mass is None else o.K + sp.diags(o.mass / s.dt ** 2)
    S0 = oracle.schur_complement(K, o.part.x1, o.part.region)
    H = S0.copy()
    if contacts.k:
        C = oracle.contact_matrix(contacts, s.n).toarray()
        H += C[np.ix_(s.region, s.region)]
    return S0, H


@pytest.mark.parametrize("name", ["config1", "small_elbow", "medium_elbow"])
def test_schur_refactor_solve_fp64(pd, name):
    if name == "config1":
        s = scenes.config1(pre_indent=0.8)
        x = s.X
        step = 0
    else:
        s = scenes.small_elbow() if name == "small_elbow" else scenes.small_elbow(h=1.0)
        x = s.X
        step = 58
    c = s.contacts(step, x)
    if c.k == 0:   # make sure the contact update is exercised
        c = scenes.sphere_contacts(s.proxies, s.X, s.X[s.proxies].mean(0), 3.0, 1e6)
    assert c.k > 0
    S0, H = _oracle_H(s, c)
    sol = _solver(pd, s)
    np.testing.assert_allclose(sol.schur(), S0, rtol=0, atol=1e-12 * np.abs(S0).max())
    sol.set_contacts(*contact_tuple(c))
    g = rng(3).normal(size=(s.m, 3)) * 1e3
    u = sol.schur_solve(g)
    res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
    assert res <= TOL, res
    uo = np.linalg.solve(H, g)
    assert np.linalg.norm(u - uo) / np.linalg.norm(uo) <= 1e3 * TOL


def _compare_step(pd, s, step, outer, inner, x0, tol):
    sol = _solver(pd, s, inner_iters=inner)
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(step))
    sol.step(outer, region_callback(s, step, x0))
    xg = sol.positions()
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    o.x = x0.copy()
    xo = o.step(outer, inner, oracle_callback(s, step), s.dirichlet_positions(step))
    err, err_node = parity_errors(xg, xo, x0)
    assert err_node <= tol, ("per node", err_node)
    return err, sol


@pytest.mark.parametrize("inner", [1, 3])
def test_one_outer_iteration_matches_oracle_config1(pd, inner):
    s = scenes.config1(pre_indent=0.6)
    x0 = s.X.copy()
    free = np.setdiff1d(np.arange(s.n), s.dirichlet)
    x0[free] += 0.05 * rng(4).normal(size=(len(free), 3))
    err, sol = _compare_step(pd, s, 0, 1, inner, x0, TOL)
    assert err <= TOL, err
    assert sol.stats()["contacts"] > 0


def test_one_outer_iteration_matches_oracle_elbow_contacts(pd):
    s = scenes.small_elbow(inner_iters=3)
    step = 52
    x0 = s.X.copy()
    err, sol = _compare_step(pd, s, step, 1, 3, x0, TOL)
    assert err <= TOL, err


def test_full_time_steps_config1_trajectory(pd):
    # 3 backward-Euler steps x 10 outer iterations with the descending sphere
    s = scenes.config1(pre_indent=0.5)
    sol = _solver(pd, s)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    for st in range(3):
        xg_prev = sol.positions()
        sol.set_dirichlet(s.dirichlet_positions(st))
        sol.step(s.outer_iters, region_callback(s, st, xg_prev))
        o.step(s.outer_iters, 1, oracle_callback(s, st), s.dirichlet_positions(st))
    xg, vg = sol.get_state()
    assert_parity(xg, o.x, s.X, 1e-8, "positions")
    assert_parity(vg, o.v, np.zeros_like(o.v), 1e-8, "velocities")


def test_errors_leave_the_handle_usable(pd):
    s = scenes.config1(nx=4, ny=4, nz=6)
    sol = _solver(pd, s)
    x_before = sol.positions()
    outside = np.setdiff1d(np.arange(s.n), s.region)[0]
    with pytest.raises(pd.PDError) as e:
        sol.set_contacts([[outside, -1, -1, -1]], [[1, 0, 0, 0]], [[0, 0, 0]], [1e6])
    assert e.value.name == "PD_ERR_CONTACT_OUTSIDE_REGION"
    # a strongly negative spring makes H indefinite: NOT_SPD, state rolled back
    r = s.region[0]
    sol.set_contacts([[r, -1, -1, -1]], [[1, 0, 0, 0]], [[0, 0, 0]], [-1e9])
    with pytest.raises(pd.PDError) as e:
        sol.step(1)
    # negative stiffness is rejected up front or reported by the factorisation
    assert e.value.name in ("PD_ERR_NOT_SPD",)
    np.testing.assert_array_equal(sol.positions(), x_before)
    sol.set_contacts(np.zeros((0, 4)), np.zeros((0, 4)), np.zeros((0, 3)), np.zeros(0))
    sol.step(1)
    assert np.all(np.isfinite(sol.positions()))


def test_state_roundtrip_and_empty_contacts(pd):
    s = scenes.config1(nx=3, ny=3, nz=5)
    sol = _solver(pd, s)
    x = s.X + 0.01
    v = np.full_like(s.X, 0.5)
    sol.set_state(x, v)
    x2, v2 = sol.get_state()
    np.testing.assert_array_equal(x2, x)
    np.testing.assert_array_equal(v2, v)
    sol.step(2)     # no contacts ever set
    assert sol.stats()["outer_done"] == 2


def test_bounded_wait_times_out_and_handle_survives(pd):
    # a device wait on a flag nothing sets gives up and reports PD_ERR_TIMEOUT
    s = scenes.config1(nx=3, ny=3, nz=5)
    sol = _solver(pd, s)
    st = pd.lib.pd_debug_wait_timeout(sol.h)
    assert pd._lib.STATUS[st] == "PD_ERR_TIMEOUT"
    assert b"gave up" in pd.lib.pd_last_error(sol.h)
    sol.step(1)                       # the context is still usable
    assert np.all(np.isfinite(sol.positions()))


def test_two_sided_springs_match_oracle(pd):
    # self-collision springs between two proxies (8-slot W rows)
    s = scenes.small_elbow(h=1.5)
    x0 = s.X.copy()
    pairs = s.info["self_pairs"](x0, gap=6.0)
    assert pairs.k > 5 and pairs.nodes.shape[1] == 8
    S0, H = _oracle_H(s, pairs)
    sol = _solver(pd, s)
    sol.set_contacts(*contact_tuple(pairs))
    g = rng(31).normal(size=(s.m, 3)) * 1e3
    u = sol.schur_solve(g)
    assert np.linalg.norm(g - H @ u) / np.linalg.norm(g) <= TOL
    # the PCG form's capacitance correction with 8-slot rows
    sol.set_precision(pd.PCG_WARM)
    u = sol.schur_solve(g)
    assert np.linalg.norm(g - H @ u) / np.linalg.norm(g) <= TOL
    assert sol.stats()["refine_iters"] <= 8
    sol.set_precision(pd.FP64)
    # one outer iteration with the pairs re-detected at every inner iteration
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(50))

    def cb(x2):
        x = x0.copy()
        x[s.region] = x2
        return contact_tuple(s.info["self_pairs"](x, gap=6.0))

    sol.step(1, cb)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(1, 1, lambda x: s.info["self_pairs"](x, gap=6.0), s.dirichlet_positions(50))
    assert_parity(sol.positions(), xo, x0, TOL)
