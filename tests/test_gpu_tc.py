"""The tcgen05 rank-K update (TMA + TMEM) against an FP64 numpy product."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu, rng

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,tol", [(0, 2.5e-3), (1, 2e-6), (2, 1.6e-2)])
@pytest.mark.parametrize("M,N", [(128, 128), (256, 384), (512, 256)])
def test_rank_k_update_matches_fp64(mode, tol, M, N):
    need_gpu()
    import torch
    import paper_2008_01541_b300 as pd
    g = rng(100 + mode)
    K = 128
    A = g.normal(size=(M, K)).astype(np.float32)
    B = g.normal(size=(N, K)).astype(np.float32)
    C = g.normal(size=(M, N)).astype(np.float32)
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    st = pd.lib.pd_tc_rank_k(mode, ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                             ctypes.c_void_p(dC.data_ptr()), M, N, K, None)
    assert st == 0
    torch.cuda.synchronize()
    out = dC.cpu().numpy().astype(np.float64)
    ref = C.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    err = np.abs(out - ref) / scale
    assert err.max() <= tol, err.max()
