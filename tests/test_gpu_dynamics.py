"""Backward-Euler mode (dt > 0, lumped mass on the diagonal of A and of
Sigma_0) on the elbow and the two-slab scenes vs the oracle."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_util import need_gpu, rng, region_callback, oracle_callback, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _run(pd, s, dt, steps, outer, prec=None):
    kw = {} if prec is None else {"precision": getattr(pd, prec)}
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, 1000.0, dt, **kw)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, 1000.0, dt)
    for st in range(steps):
        ref = sol.positions()
        sol.set_dirichlet(s.dirichlet_positions(st))
        sol.step(outer, region_callback(s, st, ref))
        o.step(outer, 1, oracle_callback(s, st), s.dirichlet_positions(st))
    return sol, o


def test_elbow_backward_euler_matches_oracle(pd):
    s = scenes.small_elbow(h=1.5)
    # start the flexion near contact so springs appear
    s0 = s.info["rest_step"]
    dpos, con = s.dirichlet_positions, s.contacts
    s.dirichlet_positions = lambda st: dpos(s0 + 10 + 2 * st)
    s.contacts = lambda st, x: con(s0 + 10 + 2 * st, x)
    sol, o = _run(pd, s, 1.0 / 30.0, 3, 5)
    x, v = sol.get_state()
    assert_parity(x, o.x, s.X, 1e-8)
    assert np.linalg.norm(v - o.v) / np.linalg.norm(o.v) <= 1e-8


def _slabs():
    s = scenes.slabs(nx=12, ny=8, nz=3, m=150)
    dpos = s.dirichlet_positions
    s.dirichlet_positions = lambda st: dpos(59)   # the jaw closed by 15 degrees from the first step
    return s


def test_slabs_backward_euler_matches_oracle(pd):
    s = _slabs()
    sol, o = _run(pd, s, 0.1, 5, 4)
    assert s.contacts(0, o.x).k > 0
    x, v = sol.get_state()
    assert_parity(x, o.x, s.X, 1e-8)
    assert np.linalg.norm(v - o.v) <= 1e-8 * max(1.0, np.linalg.norm(o.v))


def test_backward_euler_mixed_form_matches_fp64(pd):
    s = _slabs()
    a, o = _run(pd, s, 0.1, 5, 3)
    b, _ = _run(pd, s, 0.1, 5, 3, "FP32_IR")
    assert s.contacts(0, o.x).k > 0
    xa, xb = a.positions(), b.positions()
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xa - s.X) <= 1e-8
