"""The allocation-free Schur refactor + solve.

pd_schur_solve_noalloc() serves callers that may not allocate device memory
while they run (engines that reserve all GPU memory up front, arena/pool
integrations, real-time loops).  This checks, through the C ABI, that two
consecutive calls reproduce what the handle-based pd_schur_solve_dev()
computes on the same inputs, and that sizes beyond its fixed scratch are
refused.  It lives in its own file so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import scenes
from gpu_util import need_gpu, rng

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _region_contacts(s, c):
    """Contacts as region-row indices (-1 for unused slots)."""
    ridx = np.full(s.n, -1, np.int64)
    ridx[s.region] = np.arange(s.m)
    nodes = np.asarray(c.nodes, np.int64)
    idx = np.where(nodes >= 0, ridx[np.maximum(nodes, 0)], -1)
    return idx.astype(np.int32)


def test_noalloc_matches_handle_solve_twice_in_a_row():
    need_gpu()
    import torch
    import paper_2008_01541_b300 as pd
    s = scenes.config1(pre_indent=0.8)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, s.lam, s.density, s.dt)
    dev = torch.device("cuda", torch.cuda.current_device())
    sigma = torch.from_numpy(sol.schur()).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    err = ctypes.create_string_buffer(256)
    cases = [s.contacts(0, s.X), scenes.sphere_contacts(s.proxies, s.X, np.array([3.0, 6.0, 42.6]), 3.0, 5e5)]
    for call, c in enumerate(cases):
        assert c.k > 0
        sol.set_contacts(c.nodes, c.w, c.target, c.stiffness)
        g = torch.from_numpy(rng(20 + call).normal(size=(s.m, 3)) * 1e3).to(dev)
        u_ref = torch.empty_like(g)
        sol.schur_solve_dev(g, u_ref)
        torch.cuda.synchronize()
        cidx = torch.from_numpy(_region_contacts(s, c)).to(dev)
        cw = torch.from_numpy(np.ascontiguousarray(c.w)).to(dev)
        cs = torch.from_numpy(np.ascontiguousarray(c.stiffness)).to(dev)
        u = torch.full_like(g, float("nan"))
        st = pd.lib.pd_schur_solve_noalloc(_ptr(sigma), s.m, c.k, _ptr(cidx), _ptr(cw), _ptr(cs), _ptr(g),
                                           _ptr(u), ctypes.c_void_p(stream), err, 256)
        assert st == 0, err.value
        torch.cuda.synchronize()
        ur, un = u_ref.cpu().numpy(), u.cpu().numpy()
        assert np.all(np.isfinite(un))
        assert np.linalg.norm(un - ur) / np.linalg.norm(ur) <= TOL
    sol.close()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    need_gpu()
    import torch
    import paper_2008_01541_b300 as pd
    m = 1025
    dev = torch.device("cuda", torch.cuda.current_device())
    sigma = torch.eye(m, dtype=torch.float64, device=dev)
    g = torch.ones((m, 3), dtype=torch.float64, device=dev)
    u = torch.empty_like(g)
    err = ctypes.create_string_buffer(256)
    st = pd.lib.pd_schur_solve_noalloc(_ptr(sigma), m, 0, None, None, None, _ptr(g), _ptr(u), None, err, 256)
    assert st == 1 and b"1024" in err.value
