"""Parity at the benchmark's full sizes, in the configuration bench.py times:
the ~598K-tet elbow (m = 6,572) and the two-slab lips scene (m = 6,250).
Where the oracle can compute every output (local step, one outer iteration)
the comparison is element by element; the region solves are checked by
properties that hold at any size (relative residual against H = Sigma_0 + C22
in FP64 on the host)."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_util import need_gpu, rng, contact_tuple

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-10


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


@pytest.fixture(scope="module")
def elbow(pd):
    s = scenes.elbow()
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, max_refine=500)
    yield s, sol
    sol.close()


def _H(S0, s, c):
    H = S0.copy()
    ridx = np.full(s.n, -1)
    ridx[s.region] = np.arange(s.m)
    for j in range(c.k):
        for a in range(4):
            for b in range(4):
                na, nb = c.nodes[j, a], c.nodes[j, b]
                if na >= 0 and nb >= 0:
                    H[ridx[na], ridx[nb]] += c.stiffness[j] * c.w[j, a] * c.w[j, b]
    return H


def test_full_elbow_local_step(pd, elbow):
    s, sol = elbow
    x = s.X + 0.05 * rng(21).normal(size=s.X.shape)
    R, f = sol.local_step(x)
    tets = s.tets.astype(np.int64)
    Dm_inv, vol = oracle.element_precompute(s.X, tets)
    Ro = oracle.polar_rotations(oracle.deformation_gradients(x, tets, Dm_inv))
    assert np.abs(R - Ro).max() <= TOL
    fo = oracle.elastic_forces(x, Ro, tets, Dm_inv, vol, s.mu)
    assert np.abs(f - fo).max() <= TOL * np.abs(fo).max()


@pytest.mark.parametrize("prec", ["FP64", "FP32_IR", "TF32_IR", "BF16_IR", "PCG_WARM"])
def test_full_elbow_region_solve_residual(pd, elbow, prec):
    s, sol = elbow
    c = s.contacts(60, s.X)
    assert c.k > 100
    sol.set_contacts(*contact_tuple(c))
    S0 = sol.schur()
    H = _H(S0, s, c)
    g = rng(22).normal(size=(s.m, 3)) * 1e3
    sol.set_precision(getattr(pd, prec))
    u = sol.schur_solve(g)
    res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
    assert res <= TOL, (prec, res)
    sol.set_precision(pd.FP64)


def test_full_elbow_outer_iteration_matches_oracle(pd, elbow):
    s, sol = elbow
    step = 55
    x0 = s.X.copy()
    sol.set_state(x0)
    sol.set_dirichlet(s.dirichlet_positions(step))
    con = s.contacts(step, s.X)
    sol.set_contacts(*contact_tuple(con))
    sol.set_precision(pd.FP64)
    sol.step(1)
    xg = sol.positions()
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(1, 1, lambda x: con, s.dirichlet_positions(step))
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo - x0)
    assert err <= TOL, err


def test_slabs_region_solves(pd):
    s = scenes.slabs(m=6250)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, max_refine=500)
    x = s.X.copy()
    x[s.proxies] += np.array([0.0, 0.0, 0.4]) * (x[s.proxies, 2:3] < 9.25)   # lower lip pushed up
    c = s.contacts(0, x)
    assert c.k > 0
    sol.set_contacts(*contact_tuple(c))
    H = _H(sol.schur(), s, c)
    g = rng(23).normal(size=(s.m, 3)) * 1e3
    for prec in ("FP64", "FP32_IR", "BF16_IR", "PCG_WARM"):
        sol.set_precision(getattr(pd, prec))
        u = sol.schur_solve(g)
        res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
        assert res <= TOL, (prec, res)
    sol.close()
