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
from gpu_util import need_gpu, rng, contact_tuple, assert_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-10
MIXED_STEP_TOL = 5e-6   # observed 6.6e-7 (norm) / 5.1e-8 (per node) for split-TF32


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


def _tri_oracle(s):
    """The oracle's own point-triangle detection of the elbow's two sides."""
    from oracle import detect
    pa, ta, pb, tb = s.info["tri_sides"]
    gap, rmin = s.info["tri_gap"], s.info["tri_rest_min"]

    def fn(x):
        A = detect.point_triangle_springs(pa, tb, x, s.X, gap, rmin, s.stiffness)
        B = detect.point_triangle_springs(pb, ta, x, s.X, gap, rmin, s.stiffness)
        return scenes.Contacts(*(np.concatenate([A[i], B[i]]) for i in range(4)))

    return fn


def test_full_elbow_bench_step_matches_oracle(pd, elbow):
    # the step bench.py times: FP64, 1 outer x 1 inner iteration, the joint
    # closed 40 degrees, point-triangle self-contact detected on the device;
    # the oracle detects on the host and solves the full free-node system
    s, sol = elbow
    x0, fstep = scenes.closed_pose(s, 40.0)
    dpos = s.dirichlet_positions(fstep)
    pa, ta, pb, tb = s.info["tri_sides"]
    sol.set_precision(pd.FP64)
    sol.set_state(x0)
    sol.set_dirichlet(dpos)
    sol.set_detector_triangles(pa, ta, pb, tb, s.info["tri_gap"], s.info["tri_rest_min"], s.stiffness)
    sol.step(1)
    xg = sol.positions()
    # the PCG form with the capacitance correction, same step
    sol.set_precision(pd.PCG_WARM)
    sol.set_state(x0)
    sol.step(1)
    xp = sol.positions()
    pcg_iters = sol.stats()["refine_iters"]
    sol.set_precision(pd.FP64)
    sol.clear_detector()
    fn = _tri_oracle(s)
    assert fn(x0).k > 100
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(1, 1, fn, dpos)
    assert_parity(xg, xo, x0, TOL)
    assert_parity(xp, xo, x0, MIXED_STEP_TOL, "PCG_WARM + capacitance")
    assert pcg_iters <= 8, pcg_iters


def test_full_elbow_resampled_contacts_mixed_forms(pd, elbow):
    # configuration 3: the contact set resampled every step from a seeded
    # indenter schedule (springs independent of x, so no detection decision
    # can differ), split-TF32 and BF16 against the oracle, step by step from
    # the oracle's state; the error of each step is stated.  The mixed forms
    # meet a relative residual of 1e-10, which bounds the solution error by
    # about cond(H) * 1e-10 relative to the region solve's right-hand side;
    # measured against one contact step's displacement (concentrated under
    # the indenter) that is ~1e-6 here, so the bound is MIXED_STEP_TOL.
    from paper_2008_01541_b300 import warmstart as ws
    s, sol = elbow
    centres, radius = ws.indenter_path(s, seed=5, steps=2)
    dpos = s.dirichlet_positions(s.info["rest_step"])
    x = s.X.copy()
    errs = {"FP32_IR": [], "BF16_IR": []}
    for k, c in enumerate(centres):
        con = scenes.sphere_contacts(s.proxies, s.X, c, 1.3 * radius, s.stiffness)
        assert con.k > 10
        o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
        o.x = x.copy()
        xo = o.step(1, 1, lambda xx: con, dpos).copy()
        for prec in errs:
            sol.set_precision(getattr(pd, prec))
            sol.set_state(x)
            sol.set_dirichlet(dpos)
            sol.set_contacts(*contact_tuple(con))
            sol.step(1)
            assert sol.stats()["residual"] <= TOL
            e = assert_parity(sol.positions(), xo, x, MIXED_STEP_TOL, (prec, k))
            errs[prec].append(max(e))
        x = xo
    print("per-step error (worse of norm and per node):", {p: ["%.1e" % e for e in v] for p, v in errs.items()})
    sol.set_precision(pd.FP64)


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


def test_lips_12500_region_solves_and_outer_iteration(pd):
    # configuration 4 at its largest region (10%, m = 12,500): every form's
    # relative residual against H = Sigma_0 + C_22 in FP64, and one FP64
    # outer iteration against the oracle per node
    s = scenes.slabs(m=12500)
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, max_refine=500)
    x0 = s.X.copy()
    x0[s.proxies] += np.array([0.0, 0.0, 0.4]) * (x0[s.proxies, 2:3] < 9.25)   # lower lip pushed up
    c = s.contacts(0, x0)
    assert c.k > 100
    sol.set_contacts(*contact_tuple(c))
    H = _H(sol.schur(), s, c)
    g = rng(24).normal(size=(s.m, 3)) * 1e3
    for prec in ("FP64", "FP32_IR", "TF32_IR", "BF16_IR", "PCG_WARM"):
        sol.set_precision(getattr(pd, prec))
        u = sol.schur_solve(g)
        res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
        assert res <= TOL, (prec, res)
    del H
    sol.set_precision(pd.FP64)
    sol.set_state(x0)
    dpos = s.dirichlet_positions(30)
    sol.set_dirichlet(dpos)
    sol.set_contacts(*contact_tuple(c))
    sol.step(1)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(1, 1, lambda x: c, dpos)
    assert_parity(sol.positions(), xo, x0, TOL)
    sol.close()


def test_full_elbow_backward_euler_step(pd):
    # dynamic mode at scale: backward Euler on the elbow (lumped mass on the
    # diagonal of A, hence on Sigma_0's), one time step of the flexion from
    # the closed pose at rest velocity, 1 outer x 1 inner iteration with
    # point-triangle contact detected on the device, FP64 and split-TF32,
    # positions and velocities per node against the oracle
    s = scenes.elbow()
    dt, rho = 1.0 / 30.0, 1000.0
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, rho, dt, max_refine=500)
    x0, fstep = scenes.closed_pose(s, 40.0)
    v0 = 0.5 * rng(25).normal(size=x0.shape)
    v0[s.dirichlet] = 0.0
    dpos = s.dirichlet_positions(fstep + 1)
    pa, ta, pb, tb = s.info["tri_sides"]
    fn = _tri_oracle(s)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, rho, dt)
    o.x, o.v = x0.copy(), v0.copy()
    xo = o.step(1, 1, fn, dpos).copy()
    vo = o.v.copy()
    for prec, tol in (("FP64", TOL), ("FP32_IR", MIXED_STEP_TOL)):
        sol.set_precision(getattr(pd, prec))
        sol.set_state(x0, v0)
        sol.set_dirichlet(dpos)
        sol.set_detector_triangles(pa, ta, pb, tb, s.info["tri_gap"], s.info["tri_rest_min"], s.stiffness)
        sol.step(1)
        x, v = sol.get_state()
        assert_parity(x, xo, x0, tol, prec)
        # v = (x - x0) / dt for every node: the same bound scaled by 1 / dt
        assert_parity(v, vo, np.zeros_like(v), tol, prec + " v")
        sol.clear_detector()
    sol.close()


def test_lips_backward_euler_outer_iteration(pd):
    # configuration 4 (m = 6,250) in backward Euler: the region solve's
    # residual against H = Sigma_0 + C_22 (Sigma_0 now carries the x_2 mass
    # over dt^2) for every form, and one FP64 outer iteration per node
    s = scenes.slabs(m=6250)
    dt, rho = 1.0 / 30.0, 1000.0
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, rho, dt, max_refine=500)
    x0 = s.X.copy()
    x0[s.proxies] += np.array([0.0, 0.0, 0.4]) * (x0[s.proxies, 2:3] < 9.25)
    v0 = 0.3 * rng(26).normal(size=x0.shape)
    v0[s.dirichlet] = 0.0
    c = s.contacts(0, x0)
    assert c.k > 100
    sol.set_contacts(*contact_tuple(c))
    S0 = sol.schur()
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, rho, dt)
    # Sigma_0 = M_2 / dt^2 + (K_22 - K_21 (K_11 + M_1 / dt^2)^-1 K_12) and the
    # bracket is positive definite, so every diagonal entry exceeds its
    # node's mass over dt^2
    assert np.all(np.diag(S0) > o.mass[s.region] / dt ** 2)
    H = _H(S0, s, c)
    g = rng(27).normal(size=(s.m, 3)) * 1e3
    for prec in ("FP64", "FP32_IR", "BF16_IR", "PCG_WARM"):
        sol.set_precision(getattr(pd, prec))
        u = sol.schur_solve(g)
        res = np.linalg.norm(g - H @ u) / np.linalg.norm(g)
        assert res <= TOL, (prec, res)
    del H, S0
    sol.set_precision(pd.FP64)
    sol.set_state(x0, v0)
    dpos = s.dirichlet_positions(30)
    sol.set_dirichlet(dpos)
    sol.step(1)
    o.x, o.v = x0.copy(), v0.copy()
    xo = o.step(1, 1, lambda x: c, dpos)
    assert_parity(sol.positions(), xo, x0, TOL)
    sol.close()
