"""The C-ABI library: loads without a GPU, exports every declared symbol, and
its host-side partial Cholesky matches the oracle's Schur complement."""
import os
import re
import numpy as np
import pytest

import oracle
import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z_0-9]+)\s*\(", txt)) - {"pd_contact_cb", "pd_status"})


def test_library_exports_every_declared_symbol():
    import paper_2008_01541_b300 as pd
    import ctypes
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(pd.lib, n), n
        assert isinstance(getattr(pd.lib, n), ctypes._CFuncPtr)
    assert set(names) == set(pd._lib.EXPORTED)


@pytest.mark.parametrize("make", [lambda: scenes.config1(), lambda: scenes.small_elbow(),
                                  lambda: scenes.small_elbow(h=1.5, region_fraction=0.04)])
def test_host_partial_cholesky_matches_oracle_schur(make):
    import paper_2008_01541_b300 as pd
    import scipy.sparse as sp
    s = make()
    S, info = pd.host_schur(s.X, s.tets, s.region, s.dirichlet, s.mu, s.density, s.dt)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    K = o.K if o.mass is None else o.K + sp.diags(o.mass / s.dt ** 2)
    S0 = oracle.schur_complement(K, o.part.x1, o.part.region)
    assert np.abs(S - S0).max() <= 1e-12 * np.abs(S0).max()
    assert np.allclose(S, S.T, rtol=0, atol=1e-12 * np.abs(S0).max())


def test_host_setup_rejects_bad_inputs():
    import paper_2008_01541_b300 as pd
    s = scenes.tiny_cube()
    with pytest.raises(pd.PDError) as e:
        pd.host_schur(s.X, s.tets, np.concatenate([s.region, s.dirichlet[:1]]), s.dirichlet, s.mu)
    assert e.value.name == "PD_ERR_REGION"
    with pytest.raises(pd.PDError) as e:
        pd.host_schur(s.X, s.tets, np.zeros(0, np.int32), s.dirichlet, s.mu)
    assert e.value.name == "PD_ERR_REGION"
    X = s.X.copy()
    t = s.tets.copy()
    X[t[0, 3]] = X[t[0, 0]] + 0.5 * (X[t[0, 1]] - X[t[0, 0]])   # collapse one tet onto an edge
    with pytest.raises(pd.PDError) as e:
        pd.host_schur(X, t, s.region, s.dirichlet, s.mu)
    assert e.value.name == "PD_ERR_BAD_MESH"
    bad = s.tets.copy()
    bad[0, 0] = s.n + 5
    with pytest.raises(pd.PDError) as e:
        pd.host_schur(s.X, bad, s.region, s.dirichlet, s.mu)
    assert e.value.name == "PD_ERR_BAD_MESH"


def test_floating_body_schur_annihilates_translations():
    # With no Dirichlet node the PD matrix has the constant null vector, and so
    # does its Schur complement (Sigma 1 = A22 1 - A21 A11^-1 A12 1 = 0).
    import paper_2008_01541_b300 as pd
    s = scenes.tiny_cube(3, 3, 3)
    S, _ = pd.host_schur(s.X, s.tets, s.region, np.zeros(0, np.int32), s.mu)
    assert np.abs(S @ np.ones(s.m)).max() <= 1e-10 * np.abs(S).max()
