"""The allocation-free Schur refactor + solve.

pd_schur_solve_noalloc() serves callers that may not allocate device memory
while they run (engines that reserve all GPU memory up front, arena/pool
integrations, real-time loops).  This checks, through the C ABI, that two
consecutive calls reproduce what the handle-based pd_schur_solve_dev()
computes on the same inputs and solve the oracle's H = Sigma_0 + C_22; that
the largest size works and a smaller call after a larger one is not
disturbed by what the shared scratch array still holds; and that sizes
beyond the scratch, contact rows outside the region and an indefinite
matrix are refused.  It lives in its own file so that pytest collects it
last.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
        # and it solves the oracle's H = Sigma_0 + C_22 (Section 3.3) in FP64
        H = sigma.cpu().numpy() + oracle.contact_matrix(c, s.n).toarray()[np.ix_(s.region, s.region)]
        gh = g.cpu().numpy()
        assert np.linalg.norm(gh - H @ un) / np.linalg.norm(gh) <= TOL
    sol.close()


def _call(pd, sigma, m, k, cidx, cw, cs, g, u, err):
    return pd.lib.pd_schur_solve_noalloc(_ptr(sigma), m, k, _ptr(cidx), _ptr(cw), _ptr(cs), _ptr(g), _ptr(u),
                                         None, err, 256)


def _spd(m, seed):
    r = rng(seed)
    B = r.normal(size=(m, m))
    return B @ B.T / m + np.eye(m)


def test_noalloc_largest_size_then_smaller_sizes():
    # m = 1024 fills the matrix, inverse and workspace slices of the shared
    # array; the later, smaller calls must not see its leftovers
    need_gpu()
    import torch
    import paper_2008_01541_b300 as pd
    dev = torch.device("cuda", torch.cuda.current_device())
    err = ctypes.create_string_buffer(256)
    for call, m in enumerate((1024, 100, 300)):
        S = _spd(m, 30 + call)
        k = 3
        nodes = np.full((k, 4), -1, np.int32)
        nodes[:, 0] = [0, m // 2, m - 1]
        nodes[0, 1] = 1
        w = np.zeros((k, 4))
        w[:, 0] = 1.0
        w[0, :2] = [0.25, 0.75]
        c = np.array([5.0, 7.0, 11.0])
        H = S.copy()
        for j in range(k):
            for a in range(4):
                for b in range(4):
                    if nodes[j, a] >= 0 and nodes[j, b] >= 0:
                        H[nodes[j, a], nodes[j, b]] += c[j] * w[j, a] * w[j, b]
        gh = rng(40 + call).normal(size=(m, 3))
        sigma = torch.from_numpy(S).to(dev)
        g = torch.from_numpy(gh).to(dev)
        u = torch.full_like(g, float("nan"))
        st = _call(pd, sigma, m, k, torch.from_numpy(nodes).to(dev), torch.from_numpy(w).to(dev),
                   torch.from_numpy(c).to(dev), g, u, err)
        assert st == 0, (m, err.value)
        un = u.cpu().numpy()
        ref = np.linalg.solve(H, gh)
        assert np.linalg.norm(un - ref) / np.linalg.norm(ref) <= TOL, m
        assert np.linalg.norm(gh - H @ un) / np.linalg.norm(gh) <= TOL, m


def test_noalloc_refuses_bad_contacts_and_indefinite_matrices():
    need_gpu()
    import torch
    import paper_2008_01541_b300 as pd
    dev = torch.device("cuda", torch.cuda.current_device())
    err = ctypes.create_string_buffer(256)
    m = 70
    sigma = torch.from_numpy(_spd(m, 50)).to(dev)
    g = torch.ones((m, 3), dtype=torch.float64, device=dev)
    u = torch.empty_like(g)
    nodes = torch.tensor([[3, m, -1, -1]], dtype=torch.int32, device=dev)     # row m is outside the region
    w = torch.tensor([[0.5, 0.5, 0.0, 0.0]], dtype=torch.float64, device=dev)
    c = torch.tensor([1.0], dtype=torch.float64, device=dev)
    assert _call(pd, sigma, m, 1, nodes, w, c, g, u, err) == 4 and b"outside" in err.value
    S = np.eye(m)
    S[37, 37] = -1.0                                                          # indefinite
    assert _call(pd, torch.from_numpy(S).to(dev), m, 0, None, None, None, g, u, err) == 5
    assert b"pivot 37" in err.value
    # and the next good call is unaffected by the failed ones
    assert _call(pd, sigma, m, 0, None, None, None, g, u, err) == 0, err.value
    ref = np.linalg.solve(sigma.cpu().numpy(), np.ones((m, 3)))
    assert np.linalg.norm(u.cpu().numpy() - ref) / np.linalg.norm(ref) <= TOL


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
