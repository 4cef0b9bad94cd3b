"""Pins of the oracle's bi-phasic strain-limiting term (Section 5): the
projection Q onto matrices with bounded singular values, its force, the
global step with mu + mu', and the descent of the alternating iteration."""
import numpy as np
import pytest

import oracle
import scenes

LO, HI = 0.8, 1.2


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rotations(rng, k):
    A = rng.normal(size=(k, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1.0
    return Q


def test_projection_clamps_singular_values_of_a_rotated_stretch():
    rng = _rng(1)
    Ra, Rb = _rotations(rng, 5), _rotations(rng, 5)
    F = Ra @ np.diag([1.6, 1.0, 0.5]) @ np.swapaxes(Rb, 1, 2)
    want = Ra @ np.diag([1.2, 1.0, 0.8]) @ np.swapaxes(Rb, 1, 2)
    Q = oracle.strain_limit_projection(F, LO, HI)
    assert np.abs(Q - want).max() <= 1e-13


def test_projection_of_an_inverted_element_keeps_the_reflection():
    rng = _rng(2)
    Ra, Rb = _rotations(rng, 5), _rotations(rng, 5)
    F = Ra @ np.diag([1.5, 0.9, -0.3]) @ np.swapaxes(Rb, 1, 2)
    want = Ra @ np.diag([1.2, 0.9, -0.8]) @ np.swapaxes(Rb, 1, 2)
    Q = oracle.strain_limit_projection(F, LO, HI)
    assert np.abs(Q - want).max() <= 1e-13
    assert np.all(np.linalg.det(Q) < 0)


def test_projection_inside_the_bounds_is_the_identity_map():
    rng = _rng(3)
    Ra, Rb = _rotations(rng, 8), _rotations(rng, 8)
    s = rng.uniform(LO + 0.01, HI - 0.01, size=(8, 3))
    F = Ra @ (s[:, :, None] * np.swapaxes(Rb, 1, 2))
    assert np.abs(oracle.strain_limit_projection(F, LO, HI) - F).max() <= 1e-14


def test_projection_is_the_closest_point_of_the_set():
    # brute force: no sampled member of S (random orthogonal factors, any
    # sign, singular values in the bounds) is closer to F, nor any member
    # obtained by small rotations of Q's own factors
    rng = _rng(4)
    for trial in range(6):
        F = rng.normal(size=(3, 3)) * rng.uniform(0.3, 1.5)
        Q = oracle.strain_limit_projection(F[None], LO, HI)[0]
        sq = np.linalg.svd(Q, compute_uv=False)
        assert sq.min() >= LO - 1e-12 and sq.max() <= HI + 1e-12
        d0 = np.linalg.norm(F - Q)
        U = np.linalg.qr(rng.normal(size=(4000, 3, 3)))[0]
        V = np.linalg.qr(rng.normal(size=(4000, 3, 3)))[0]
        s = rng.uniform(LO, HI, size=(4000, 3))
        cand = U @ (s[:, :, None] * np.swapaxes(V, 1, 2))
        assert d0 <= np.linalg.norm(F[None] - cand, axis=(1, 2)).min() + 1e-12
        Uq, sq, Vqt = np.linalg.svd(Q)
        for _ in range(300):
            a, b = rng.normal(size=(2, 3)) * 1e-3
            Ka = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
            Kb = np.array([[0, -b[2], b[1]], [b[2], 0, -b[0]], [-b[1], b[0], 0]])
            ds = np.clip(sq + rng.normal(size=3) * 1e-3, LO, HI)
            Qp = (Uq @ (np.eye(3) + Ka)) @ np.diag(ds) @ ((np.eye(3) + Kb) @ Vqt)
            Up, _, Vpt = np.linalg.svd(Qp)
            Qp = Up @ np.diag(np.clip(np.linalg.svd(Qp, compute_uv=False), LO, HI)) @ Vpt
            assert d0 <= np.linalg.norm(F - Qp) + 1e-12


def _energy_at(o, x):
    all_e = np.arange(len(o.tets))
    return o.energy(x, o.rotations(x, all_e), Q=o.projections(x, all_e))


def test_biphasic_force_is_minus_gradient_of_the_minimised_energy():
    # Danskin: with R and Q the exact minimisers, -dE'/dx equals the force at
    # fixed (R, Q); a wrong Q would add a dQ/dx term and break the match
    X, tets, _ = scenes.grid_mesh(2, 2, 3)
    X = X + 0.05 * _rng(5).normal(size=X.shape)
    tets = tets.astype(np.int64)
    o = oracle.OracleSolver(X, tets, np.zeros(0, np.int64), np.zeros(0, np.int64), 1e4, mu_prime=5e4,
                            sigma_min=LO, sigma_max=HI)
    rng = _rng(6)
    x = X * np.array([1.25, 0.85, 1.0]) + 0.05 * rng.normal(size=X.shape)
    all_e = np.arange(len(tets))
    R, Q = o.rotations(x, all_e), o.projections(x, all_e)
    sv = np.linalg.svd(oracle.deformation_gradients(x, tets, o.Dm_inv), compute_uv=False)
    assert (sv > HI).any() and (sv < LO).any()
    f = (oracle.elastic_forces(x, R, tets, o.Dm_inv, o.vol, o.mu)
         + oracle.elastic_forces(x, Q, tets, o.Dm_inv, o.vol, o.mu_prime))
    for _ in range(5):
        d = rng.normal(size=x.shape)
        eps = 1e-6
        fd = -(_energy_at(o, x + eps * d) - _energy_at(o, x - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(f * d)) <= 1e-5 * np.abs(f * d).sum()


def test_biphasic_global_step_is_force_equilibrium():
    s = scenes.config1(pre_indent=0.6, nx=3, ny=3, nz=6)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, mu_prime=4 * s.mu,
                            sigma_min=0.95, sigma_max=1.05)
    rng = _rng(7)
    x = s.X.copy()
    x[o.part.free] += 0.15 * rng.normal(size=(len(o.part.free), 3))
    all_e = np.arange(s.E)
    R, Q = o.rotations(x, all_e), o.projections(x, all_e)
    con = s.contacts(0, x)
    x1 = o.full_solve(x, R, con, None, Q)
    f = (oracle.elastic_forces(x1, R, o.tets, o.Dm_inv, o.vol, o.mu)
         + oracle.elastic_forces(x1, Q, o.tets, o.Dm_inv, o.vol, o.mu_prime)
         + oracle.contact_forces(con, x1))
    scale = np.abs(oracle.elastic_forces(x, R, o.tets, o.Dm_inv, o.vol, o.mu)).max()
    assert np.abs(f[o.part.free]).max() <= 1e-9 * scale


def test_biphasic_energy_never_increases_across_local_and_global_steps():
    s = scenes.config1(pre_indent=0.6, nx=3, ny=3, nz=6)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, mu_prime=10 * s.mu,
                            sigma_min=0.97, sigma_max=1.03)
    rng = _rng(8)
    x = s.X.copy()
    x[o.part.free] += 0.15 * rng.normal(size=(len(o.part.free), 3))
    con = s.contacts(0, x)
    assert con.k > 0
    all_e = np.arange(s.E)
    R, Q = o.rotations(x, all_e), o.projections(x, all_e)
    last = o.energy(x, R, con, Q=Q)
    for _ in range(6):
        R, Q = o.rotations(x, all_e), o.projections(x, all_e)      # local step
        e = o.energy(x, R, con, Q=Q)
        assert e <= last * (1 + 1e-12)
        last = e
        x = o.full_solve(x, R, con, None, Q)                       # global step
        e = o.energy(x, R, con, Q=Q)
        assert e <= last * (1 + 1e-12)
        last = e


def test_unit_bounds_reduce_to_plain_pd_with_mu_plus_mu_prime():
    # sigma_min = sigma_max = 1 makes Q the polar rotation of a non-inverted F,
    # so the bi-phasic step is the plain step with stiffness mu + mu'
    s = scenes.config1(pre_indent=0.6, nx=3, ny=3, nz=6)
    mu, mp = s.mu, 3 * s.mu
    a = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, mu, mu_prime=mp, sigma_min=1.0, sigma_max=1.0)
    b = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, mu + mp)
    fn = lambda x: s.contacts(0, x)   # noqa: E731
    xa = a.step(3, 2, fn).copy()
    xb = b.step(3, 2, fn).copy()
    assert np.linalg.norm(xa - xb) <= 1e-10 * np.linalg.norm(xb - s.X)


def test_unbounded_set_keeps_the_plain_pd_equilibrium():
    # with S = all matrices the mu' term has zero energy; the iteration with
    # mu' > 0 (a different system matrix) must converge to the same x
    s = scenes.config1(pre_indent=0.8, nx=3, ny=3, nz=5)
    con = s.contacts(0, s.X)
    assert con.k > 0
    fn = lambda x: con   # noqa: E731
    a = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, mu_prime=2 * s.mu)
    b = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    for _ in range(60):
        a.step(20, 1, fn)
        b.step(20, 1, fn)
        d = np.linalg.norm(a.x - b.x) / np.linalg.norm(b.x - s.X)
        if d < 1e-7:
            break
    assert d < 1e-7, d
