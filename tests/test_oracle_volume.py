"""Pins of the oracle's PD volume term kappa ||F - T||^2 (the PD form of the
lambda term of Eq. 1): the projection T onto matrices with determinant in
[det_min, det_max], its agreement with the lambda term at small strain, its
force, the global step with mu + kappa and the descent of the alternating
iteration."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from oracle import pd_oracle
import scenes


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rotations(rng, k):
    A = rng.normal(size=(k, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1.0
    return Q


def _expm_traceless(rng, scale):
    A = scale * rng.normal(size=(3, 3))
    A -= np.trace(A) / 3.0 * np.eye(3)
    w, V = np.linalg.eig(A)
    return np.real(V @ np.diag(np.exp(w)) @ np.linalg.inv(V))


def test_inside_the_bounds_is_the_identity_map():
    rng = _rng(1)
    Ra, Rb = _rotations(rng, 6), _rotations(rng, 6)
    s = np.array([[1.05, 1.0, 0.95], [1.2, 0.9, 0.95], [1.0, 1.0, 1.0],
                  [0.98, 0.97, 0.96], [1.1, 1.0, 0.92], [1.01, 1.01, 1.01]])
    F = Ra @ (s[:, :, None] * np.eye(3)) @ np.swapaxes(Rb, 1, 2)
    assert np.all((np.linalg.det(F) >= 0.85) & (np.linalg.det(F) <= 1.15))
    T = oracle.volume_projection(F, 0.85, 1.15)
    assert np.array_equal(T, F)


@pytest.mark.parametrize("scale,lo,hi,want", [
    (0.5, 1.0, 1.0, 1.0), (0.8, 1.0, 1.0, 1.0), (1.3, 1.0, 1.0, 1.0), (1.8, 1.0, 1.0, 1.0),
    (0.5, 0.8, 1.2, 0.8 ** (1 / 3)), (1.3, 0.8, 1.2, 1.2 ** (1 / 3)),
])
def test_isotropic_stretch_closed_form(scale, lo, hi, want):
    # F = s Q: the nearest matrix with determinant v is v^(1/3) Q
    Q = _rotations(_rng(2), 4)
    T = oracle.volume_projection(scale * Q, lo, hi)
    assert np.abs(T - want * Q).max() <= 1e-14


def test_inverted_element_is_restored_to_the_bound():
    # F = diag(1, 1, -0.2): tau solves (tau_i - s_i) tau_i = -c with the same
    # c for every i and tau_1 tau_2 tau_3 = 1 (Lagrange stationarity)
    T = oracle.volume_projection(np.diag([1.0, 1.0, -0.2]), 1.0, 1.0)
    tau = np.diag(T)
    assert np.abs(T - np.diag(tau)).max() == 0.0
    assert tau[0] == tau[1] and tau[2] > 0.0
    assert abs(np.prod(tau) - 1.0) <= 1e-14
    c = (tau - np.array([1.0, 1.0, -0.2])) * tau
    assert np.ptp(c) <= 1e-14


def test_determinant_meets_the_violated_bound_and_singular_vectors_are_kept():
    rng = _rng(3)
    n = 300
    Ra, Rb = _rotations(rng, n), _rotations(rng, n)
    s = np.sort(rng.uniform(0.3, 1.7, size=(n, 3)), axis=1)[:, ::-1]
    s[: n // 5, 2] *= -0.5           # some inverted elements
    F = Ra @ (s[:, :, None] * np.eye(3)) @ np.swapaxes(Rb, 1, 2)
    lo, hi = 0.9, 1.1
    T = oracle.volume_projection(F, lo, hi)
    d, dt = np.linalg.det(F), np.linalg.det(T)
    out = (d < lo) | (d > hi)
    assert out.sum() > n // 2
    want = np.where(d < lo, lo, hi)
    assert np.abs(dt[out] - want[out]).max() <= 1e-13
    # T = Ra diag(tau) Rb^T with every tau_i > 0 and ordered like s
    D = np.swapaxes(Ra, 1, 2) @ T @ Rb
    off = D - D * np.eye(3)
    assert np.abs(off).max() <= 1e-13
    tau = np.diagonal(D, axis1=1, axis2=2)
    assert np.all(tau[out] > 0)
    assert np.all(np.diff(tau[out], axis=1) <= 1e-13)


def test_nearest_point_against_a_library_qp_and_perturbations():
    # contraction, inversion and expansions up to 1.6x: the oracle's T is at
    # least as close to F as every other matrix with det = v that a library
    # QP (several starts, collapsed and sign-flipped ones included) finds,
    # and as every perturbation T exp(A), exp(A) T with tr A = 0
    rng = _rng(4)
    for k in range(40):
        s = np.sort(rng.uniform(0.4, 1.6, size=3))[::-1].copy()
        if k % 4 == 0:
            s[2] = -rng.uniform(0.05, 0.5)
        v = rng.choice([0.9, 1.0, 1.1])
        Ra, Rb = _rotations(rng, 2)
        F = Ra @ np.diag(s) @ Rb.T
        d = np.linalg.det(F)
        if abs(d - v) < 1e-3:
            continue
        T = oracle.volume_projection(F, v, v)
        dist = np.linalg.norm(F - T)
        best = np.inf
        starts = [np.abs(s), np.full(3, v ** (1 / 3)), np.array([s[0], s[1], v / (s[0] * s[1])]),
                  np.array([-abs(s[0]), -abs(s[1]), v / (s[0] * s[1])]), rng.uniform(0.2, 2.0, 3)]
        for x0 in starts:
            r = minimize(lambda t: np.sum((t - s) ** 2), x0,
                         constraints=[{"type": "eq", "fun": lambda t: np.prod(t) - v}],
                         method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
            if r.success and abs(np.prod(r.x) - v) < 1e-8:
                best = min(best, np.sqrt(r.fun))
        assert dist <= best + 1e-7, (s, v, dist, best)
        for _ in range(50):
            E = _expm_traceless(rng, 0.05)
            for Tp in (T @ E, E @ T):
                assert np.linalg.norm(F - Tp) >= dist - 1e-12


def test_small_strain_agrees_with_the_lambda_term():
    # (3 lambda / 2) ||F - T||^2 / ((lambda / 2) tr^2(S - I)) -> 1 as the
    # strain goes to zero (the error is first order in the strain)
    rng = _rng(5)
    R = _rotations(rng, 1)[0]
    E = rng.normal(size=(3, 3))
    E = 0.5 * (E + E.T)
    E += 0.3 * np.eye(3)           # a volume change
    prev = np.inf
    for eps in (1e-2, 1e-3, 1e-4):
        F = R @ (np.eye(3) + eps * E)
        T = oracle.volume_projection(F, 1.0, 1.0)
        ratio = 3.0 * np.sum((F - T) ** 2) / np.trace(eps * E) ** 2
        assert abs(ratio - 1.0) < 30 * eps
        assert abs(ratio - 1.0) < prev
        prev = abs(ratio - 1.0)


def test_branch_end_for_a_large_isotropic_stretch():
    # 3x in every direction: no point of det = 1 lies on the principal
    # branch, T is its end (each singular value halved).  At the branch end
    # tau_i = (s_i + sqrt(s_i^2 - s_3^2)) / 2 turns rounding-level differences
    # between equal singular values into ~sqrt(eps) ones
    Q = _rotations(_rng(6), 1)[0]
    T = oracle.volume_projection(3.0 * Q, 1.0, 1.0)
    assert np.abs(T - 1.5 * Q).max() <= 1e-7
    T = oracle.volume_projection(np.diag([3.0, 3.0, 3.0]), 1.0, 1.0)
    assert np.abs(T - 1.5 * np.eye(3)).max() <= 1e-15


def _small(pre=0.6):
    return scenes.config1(pre_indent=pre, nx=3, ny=3, nz=6)


def test_volume_force_is_minus_gradient_at_fixed_targets():
    s = _small()
    kappa = 5 * s.mu
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, kappa=kappa, det_min=1.0, det_max=1.0)
    rng = _rng(7)
    x = s.X + 0.1 * rng.normal(size=s.X.shape)
    all_e = np.arange(s.E)
    R, T = o.rotations(x, all_e), o.volume_targets(x, all_e)
    f = (oracle.elastic_forces(x, R, o.tets, o.Dm_inv, o.vol, o.mu)
         + oracle.elastic_forces(x, T, o.tets, o.Dm_inv, o.vol, kappa))
    for (i, c) in [(7, 0), (40, 1), (100, 2), (s.n - 3, 0)]:
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        g = (o.energy(xp, R, T=T) - o.energy(xm, R, T=T)) / (2 * h)
        assert abs(g + f[i, c]) <= 1e-6 * max(1.0, abs(f[i, c]))


def test_volume_global_step_is_force_equilibrium():
    s = _small()
    kappa = 5 * s.mu
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, kappa=kappa, det_min=0.95, det_max=1.05)
    rng = _rng(8)
    x = s.X.copy()
    x[o.part.free] += 0.1 * rng.normal(size=(len(o.part.free), 3))
    con = s.contacts(0, x)
    assert con.k > 0
    all_e = np.arange(s.E)
    R, T = o.rotations(x, all_e), o.volume_targets(x, all_e)
    x1 = o.full_solve(x, R, con, None, None, T)
    f = (oracle.elastic_forces(x1, R, o.tets, o.Dm_inv, o.vol, o.mu)
         + oracle.elastic_forces(x1, T, o.tets, o.Dm_inv, o.vol, kappa)
         + oracle.contact_forces(con, x1))
    scale = np.abs(oracle.elastic_forces(x, R, o.tets, o.Dm_inv, o.vol, o.mu)).max()
    assert np.abs(f[o.part.free]).max() <= 1e-9 * scale


def test_volume_energy_never_increases_across_local_and_global_steps():
    s = _small()
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, kappa=10 * s.mu, det_min=1.0, det_max=1.0)
    rng = _rng(9)
    x = s.X.copy()
    x[o.part.free] += 0.15 * rng.normal(size=(len(o.part.free), 3))
    con = s.contacts(0, x)
    all_e = np.arange(s.E)
    R, T = o.rotations(x, all_e), o.volume_targets(x, all_e)
    last = o.energy(x, R, con, T=T)
    for _ in range(6):
        R, T = o.rotations(x, all_e), o.volume_targets(x, all_e)      # local step
        e = o.energy(x, R, con, T=T)
        assert e <= last * (1 + 1e-12)
        last = e
        x = o.full_solve(x, R, con, None, None, T)                     # global step
        e = o.energy(x, R, con, T=T)
        assert e <= last * (1 + 1e-12)
        last = e


def test_wide_bounds_keep_the_plain_pd_equilibrium():
    # with bounds no element reaches, the kappa term has zero energy; the
    # iteration with kappa > 0 (a different system matrix) converges to the
    # same x as plain PD
    s = scenes.config1(pre_indent=0.8, nx=3, ny=3, nz=5)
    con = s.contacts(0, s.X)
    fn = lambda x: con   # noqa: E731
    a = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, kappa=2 * s.mu, det_min=1e-3, det_max=1e3)
    b = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    for _ in range(60):
        a.step(20, 1, fn)
        b.step(20, 1, fn)
        d = np.linalg.norm(a.x - b.x) / np.linalg.norm(b.x - s.X)
        if d < 1e-7:
            break
    assert d < 1e-7, d


def test_volume_term_reduces_volume_change_under_contact():
    # the same indentation loses less volume the larger kappa is (the reason
    # for the term): mean |det F - 1| over the elements after the same steps
    s = scenes.config1(pre_indent=0.8, nx=3, ny=3, nz=5)
    con = s.contacts(0, s.X)
    fn = lambda x: con   # noqa: E731
    out = []
    for kappa in (0.0, 10 * s.mu, 100 * s.mu):
        o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, kappa=kappa)
        for _ in range(4):
            o.step(10, 1, fn)
        F = oracle.deformation_gradients(o.x, o.tets, o.Dm_inv)
        out.append(np.abs(np.linalg.det(F) - 1.0).mean())
    assert out[0] > out[1] > out[2], out


def test_signed_svd_reconstructs_and_marks_inversion():
    rng = _rng(10)
    F = rng.normal(size=(50, 3, 3))
    U, s, Vt = pd_oracle.signed_svd(F)
    assert np.abs((U * s[:, None, :]) @ Vt - F).max() <= 1e-13
    assert np.all(np.abs(np.linalg.det(U) - 1) <= 1e-13)
    assert np.all(np.abs(np.linalg.det(Vt) - 1) <= 1e-13)
    assert np.array_equal(s[:, 2] < 0, np.linalg.det(F) < 0)
