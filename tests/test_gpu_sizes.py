"""Region sizes at and around the tile boundaries of the dense kernels (FP64
tiles of 64, low-precision tiles of 128, 32-row panel slices), every form,
against the oracle's H = Sigma_0 + C_22 and one outer iteration vs the oracle.
Sizes 300 and 400 give the low-precision preconditioner three and four block
rows, so its off-chain block products run as well."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import scenes
from scenes.mesh import jitter_interior
from gpu_util import need_gpu, rng, contact_tuple, assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10
SIZES = [1, 3, 17, 63, 64, 65, 127, 128, 129, 200, 300, 400]


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _scene(m):
    # 8 x 8 x 10 cubes, bottom fixed; the region is the m highest free nodes
    X, tets, g = scenes.grid_mesh(8, 8, 10, 1.0)
    X = jitter_interior(X, tets, 0.1, 3)
    dirichlet = np.nonzero(g[:, 2] == 0)[0].astype(np.int32)
    order = np.lexsort((np.arange(len(X)), -X[:, 2]))
    region = np.sort(order[:m]).astype(np.int32)
    proxies = region
    s = scenes.Scene("sizes", X, tets.astype(np.int32), dirichlet, region, proxies, dt=0.0)
    c = scenes.sphere_contacts(region, X, X[region].mean(0) + np.array([0, 0, 1.5]), 2.5, 1e6)
    return s, c


def _oracle_H(s, c):
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    S0 = oracle.schur_complement(o.K, o.part.x1, o.part.region)
    H = S0.copy()
    if c.k:
        H += oracle.contact_matrix(c, len(s.X)).toarray()[np.ix_(s.region, s.region)]
    return H


@pytest.mark.parametrize("m", SIZES)
def test_every_form_solves_ragged_regions(pd, m):
    s, c = _scene(m)
    H = _oracle_H(s, c)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, max_refine=500)
    sol.set_contacts(*contact_tuple(c))
    g = rng(60 + m).normal(size=(m, 3)) * 1e3
    for p in ["FP64", "FP32_IR", "TF32_IR", "BF16_IR", "PCG_WARM"]:
        sol.set_precision(getattr(pd, p))
        u = sol.schur_solve(g)
        res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
        assert res <= TOL, (m, p, res)


@pytest.mark.parametrize("m", [1, 65, 129])
def test_outer_iteration_ragged_region_matches_oracle(pd, m):
    s, c = _scene(m)
    x0 = s.X.copy()
    free = np.setdiff1d(np.arange(len(s.X)), s.dirichlet)
    x0[free] += 0.02 * rng(70 + m).normal(size=(len(free), 3))
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, inner_iters=2)
    sol.set_state(x0)
    sol.set_contacts(*contact_tuple(c))
    sol.step(1)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(1, 2, lambda x: c, s.X[s.dirichlet])
    assert_parity(sol.positions(), xo, x0, TOL, m)
