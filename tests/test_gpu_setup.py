"""The numeric phase of the setup on the device (Section 3.1, Eq. 9): the
multifrontal partial Cholesky whose Schur complement Sigma_0 the solver
starts from, against the oracle's Schur complement of the same matrix and
against the library's host factorisation of the same symbolic analysis;
small fronts (one CTA each), large fronts (the blocked FP64 tile factor on
padded fronts), backward Euler's mass term, the bi-phasic and volume weights,
the full-size elbow, and a matrix that is not positive definite."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import scenes
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _device_schur(pd, s, **kw):
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, s.density, s.dt, **kw)
    S = sol.schur()
    sol.close()
    return S


@pytest.mark.parametrize("make", [lambda: scenes.config1(), lambda: scenes.small_elbow(),
                                  lambda: scenes.small_elbow(h=1.0), lambda: scenes.slabs(nx=40, ny=20, nz=5, m=600)])
def test_device_schur_matches_oracle(pd, make):
    s = make()
    S = _device_schur(pd, s)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    K = o.K if o.mass is None else o.K + sp.diags(o.mass / s.dt ** 2)
    S0 = oracle.schur_complement(K, o.part.x1, o.part.region)
    assert np.abs(S - S0).max() <= 1e-12 * np.abs(S0).max()
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S0).max()   # the beta block's sums are not ordered alike


@pytest.mark.parametrize("kw", [dict(), dict(mu_prime=3.0e4), dict(kappa=6.0e4, det_min=0.95, det_max=1.05)])
def test_device_schur_matches_host_factorisation(pd, kw):
    # backward Euler (mass / dt^2 on the diagonal) with the element weights
    # 2 (mu + mu' + kappa) Vol: the same symbolic analysis, factored on the
    # device and on the host
    s = scenes.small_elbow(h=1.0)
    s.density, s.dt = 1000.0, 1.0 / 30.0
    S = _device_schur(pd, s, **kw)
    Sh, _ = pd.host_schur(s.X, s.tets, s.region, s.dirichlet, s.mu, s.density, s.dt,
                          mu_prime=kw.get("mu_prime", 0.0), kappa=kw.get("kappa", 0.0))
    assert np.abs(S - Sh).max() <= 1e-12 * np.abs(Sh).max()


def test_device_schur_full_size_elbow(pd):
    # 598K tets, m = 6,572: fronts up to order ~6,900 (padded large fronts)
    s = scenes.elbow()
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, 0.0, 0.0)
    S = sol.schur()
    setup_ms = sol.stats()["setup_ms"]
    sol.close()
    Sh, info = pd.host_schur(s.X, s.tets, s.region, s.dirichlet, s.mu)
    assert np.abs(S - Sh).max() <= 1e-12 * np.abs(Sh).max()
    print("setup %.0f ms (host: %s)" % (setup_ms, info))


def test_interior_not_positive_definite_is_reported(pd):
    # a second body with no Dirichlet node and no region node: its interior
    # block is singular, which the device factorisation must report
    s = scenes.config1(nx=3, ny=3, nz=4)
    shift = np.array([100.0, 0.0, 0.0])
    X = np.vstack([s.X, s.X + shift])
    tets = np.vstack([s.tets, s.tets + s.n])
    with pytest.raises(pd.PDError) as e:
        pd.Solver(X, tets, s.region, s.dirichlet, s.mu, 0.0, 0.0, 0.0)
    assert e.value.name == "PD_ERR_NOT_SPD"
