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


def test_learned_start_by_starting_point(pd):
    # configuration 5 in small: region solves recorded by the method along
    # seeded indenter paths, the network trained on them, then held-out
    # paths run with PCG from each starting point (zero, previous solution,
    # z0, network).  A start is kept only when it is closer to the solution
    # than zero in the H-norm (the energy PCG minimises); with penalty
    # springs of 1e6 an error at a spring node costs ~1e6 / diag(Sigma_0)
    # more than elsewhere, so starts that are good in the Euclidean norm are
    # routinely worse than zero in the H-norm
    from paper_2008_01541_b300 import warmstart as ws
    s = scenes.small_elbow(h=1.5)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, precision=pd.FP32_IR, inner_iters=2,
                    max_refine=400)
    sol.set_dirichlet(s.dirichlet_positions(s.info["rest_step"]))
    x0, v0 = sol.get_state()
    sol.mlp_set_params(ws.he_init(0))
    sol.mlp_set_loss(1)
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
    err_net, err_zero = sol.mlp_eval()
    sol.mlp_record(0)
    # beyond the contact-free response z0, the network predicts most of the rest
    assert err_net < 0.3 * err_zero, (err_net, err_zero)
    sol.set_precision(pd.PCG_WARM)
    total, rejected = {}, {}
    for src in (0, 1, 3, 2):
        sol.set_state(x0, v0)
        sol.set_warm_start(src)
        r0 = sol.stats()["starts_rejected"]
        total[src] = sum(ws.run_path(sol, s, centres, radius))   # every solve reached 1e-10
        rejected[src] = sol.stats()["starts_rejected"] - r0
    print("held-out error of the correction after z0: network %.4f of the z0 start" % (err_net / err_zero))
    print("PCG iterations by start (0 zero, 1 previous, 3 z0, 2 network):", total,
          "starts replaced by zero:", rejected)
    assert rejected[0] == 0
    # a start is never worse than the cold start in the H-norm, so no start
    # costs materially more iterations than zero
    for src in (1, 3, 2):
        assert total[src] <= 1.1 * total[0] + 2, (src, total)
