"""The learned warm start: hand-written forward/backward kernels vs the FP64
oracle, training on solves the method generates, and what the network gains
as a PCG starting point over starting without it."""
import numpy as np
import pytest

import scenes
from oracle import mlp
from gpu_util import need_gpu, rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_2008_01541_b300 as pd
    return pd


def _round_weights(p):
    """BF16 weights, FP32 biases: what the device computes with."""
    out = np.array(p, dtype=np.float64)
    q = 0
    for n, k in mlp.SIZES:
        out[q:q + n * k] = mlp.bf16_round(out[q:q + n * k])
        q += n * k + n
    return out


# Per-layer bound of the device gradients against the FP64 reference that
# stores the same intermediates in BF16 (activations and dL/dZ, where the
# device does): both round the same values, so they differ by FP32 against
# FP64 accumulation (~256 x 2^-24 relative per product) and the rare BF16
# rounding it flips (one BF16 spacing, 2^-8, on single entries).  A wrong
# bias gradient or ReLU mask in any layer moves its block by O(1).
GRAD_MAX_REL = 1e-3      # observed <= 3e-4 per block


def test_gradients_match_the_fp64_oracle(pd):
    s = scenes.config1(nx=3, ny=3, nz=5)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu)
    g = rng(11)
    p = mlp.init_params(5)
    p[np.arange(len(p)) % 7 == 0] += 0.01            # nonzero biases too
    X = g.normal(size=(300, 14))
    T = 0.5 * g.normal(size=(300, 3))
    sol.mlp_set_params(p.astype(np.float32))
    np.testing.assert_array_equal(sol.mlp_get_params(), p.astype(np.float32))
    loss_g, grad_g = sol.mlp_loss_grad(X.astype(np.float32), T.astype(np.float32))
    loss_o, grad_o = mlp.loss_grad(_round_weights(p.astype(np.float32)), mlp.bf16_round(X), T.astype(np.float32),
                                   store=mlp.bf16_round)
    assert abs(loss_g - loss_o) <= 1e-4 * loss_o
    q = 0
    worst = []
    for n, k in mlp.SIZES:
        for size in (n * k, n):
            a, b = grad_g[q:q + size], grad_o[q:q + size]
            rel = np.abs(a - b).max() / np.abs(b).max()
            worst.append(((n, k, size), rel))
            assert rel <= GRAD_MAX_REL, (n, k, size, rel)
            q += size
    print("per-block max relative gradient error:", ["%s %.1e" % w for w in worst])


def test_learned_start_cuts_pcg_iterations(pd):
    from paper_2008_01541_b300 import warmstart as ws
    s = scenes.small_elbow(h=1.5)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, precision=pd.FP32_IR, inner_iters=2,
                    max_refine=400)
    sol.set_dirichlet(s.dirichlet_positions(s.info["rest_step"]))
    x0, v0 = sol.get_state()
    sol.mlp_set_params(ws.he_init(0))
    sol.mlp_record(400)
    centres, radius = ws.indenter_path(s, seed=1, steps=200)
    ws.run_path(sol, s, centres, radius)
    first = sol.mlp_train(1, batch=1024, lr=1e-3, seed=2)
    last = sol.mlp_train(3000, batch=1024, lr=1e-3, seed=3)
    assert last < 0.5 * first, (first, last)
    # held-out solves from a new indenter path, recorded by the method itself
    sol.mlp_record(100)
    centres, radius = ws.indenter_path(s, seed=99, steps=25)
    sol.set_state(x0, v0)
    ws.run_path(sol, s, centres, radius)
    mse_net, mse_zero = sol.mlp_eval()
    sol.mlp_record(0)
    # beyond the contact-free response z0, the network predicts a good part of the rest
    assert mse_net < 0.7 * mse_zero, (mse_net, mse_zero)
    # PCG iterations to 1e-10 by starting point, reported (the contact-free
    # preconditioner leaves one outlier eigenvalue per active spring, which
    # bounds what any starting point can save)
    sol.set_precision(pd.PCG_WARM)
    total = {}
    for src in (0, 1, 3, 2):
        sol.set_state(x0, v0)
        sol.set_warm_start(src)
        total[src] = sum(ws.run_path(sol, s, centres, radius))
    print("held-out squared error of the correction after z0: network %.3f of the z0 start" % (mse_net / mse_zero))
    print("PCG iterations by start (0 zero, 1 previous, 3 z0, 2 network):", total)
