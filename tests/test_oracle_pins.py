"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-derive a value by calling the oracle's own routine a second
way: each checks a closed form, an invariant, a finite difference of the
energy, or a literal dense re-statement of Algorithm 1.
"""
import os
import numpy as np
import pytest

import oracle
import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def _random_rotations(rng, k):
    q = rng.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], 1)


def _read_gold(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b = line.split("|")
        rows.append((np.array(a.split(), float), np.array(b.split(), float)))
    return rows


# ---------------------------------------------------------------- local step
def test_polar_closed_form_diagonal():
    for a, r in _read_gold("polar_closed_form.txt"):
        R = oracle.polar_rotations(np.diag(a)[None])[0]
        np.testing.assert_allclose(R, np.diag(r), atol=1e-14)


def test_polar_is_rotation_and_identity():
    rng = _rng(1)
    F = rng.normal(size=(2000, 3, 3))
    R = oracle.polar_rotations(F)
    err = np.abs(np.einsum("eji,ejk->eik", R, R) - np.eye(3)).max()
    assert err <= 1e-13
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-13)
    I = oracle.polar_rotations(np.eye(3)[None])[0]
    np.testing.assert_allclose(I, np.eye(3), atol=1e-15)


def test_polar_of_rotation_times_spd_is_the_rotation():
    rng = _rng(2)
    Q = _random_rotations(rng, 500)
    B = rng.normal(size=(500, 3, 3))
    S = np.einsum("eij,ekj->eik", B, B) + 0.5 * np.eye(3)
    R = oracle.polar_rotations(Q @ S)
    np.testing.assert_allclose(R, Q, atol=1e-11)


def test_polar_minimises_psi_hat():
    # Psi_hat(F, R) <= Psi_hat(F, R') for 10^4 random rotations R' (Eq. 2, Section 2.2)
    rng = _rng(3)
    Rp = _random_rotations(rng, 10000)
    for trial in range(6):
        F = rng.normal(size=(3, 3))
        if trial % 2:
            F[:, 0] *= -1.0          # inverted element
        R = oracle.polar_rotations(F[None])[0]
        best = np.sum((F - R) ** 2)
        others = np.sum((F[None] - Rp) ** 2, axis=(1, 2))
        assert best <= others.min() + 1e-12


# ---------------------------------------------------------------- energy, forces, matrix
def _small_mesh(seed=0):
    X, tets, _ = scenes.grid_mesh(2, 2, 3)
    X = X + 0.05 * _rng(seed).normal(size=X.shape)
    return X, tets.astype(np.int64)


def test_volumes_and_mass_sum_to_box():
    X, tets, _ = scenes.grid_mesh(3, 4, 5, h=0.5)
    _, vol = oracle.element_precompute(X, tets.astype(np.int64))
    assert abs(vol.sum() - 3 * 4 * 5 * 0.125) < 1e-12
    m = oracle.lumped_mass(tets.astype(np.int64), vol, 1000.0, len(X))
    assert abs(m.sum() - 1000.0 * 7.5) < 1e-9


def test_forces_are_minus_energy_gradient():
    X, tets = _small_mesh()
    rng = _rng(4)
    Dm_inv, vol = oracle.element_precompute(X, tets)
    x = X + 0.2 * rng.normal(size=X.shape)
    R = _random_rotations(rng, len(tets))
    mu = 1e4
    f = oracle.elastic_forces(x, R, tets, Dm_inv, vol, mu)
    for _ in range(5):
        d = rng.normal(size=x.shape)
        eps = 1e-3
        ep = oracle.pd_energy(x + eps * d, R, tets, Dm_inv, vol, mu)
        em = oracle.pd_energy(x - eps * d, R, tets, Dm_inv, vol, mu)
        fd = -(ep - em) / (2 * eps)          # exact for a quadratic up to rounding
        assert abs(fd - np.sum(f * d)) <= 1e-8 * max(1.0, abs(fd))


def test_matrix_is_hessian_and_rhs_is_projection():
    X, tets = _small_mesh(1)
    rng = _rng(5)
    Dm_inv, vol = oracle.element_precompute(X, tets)
    n = len(X)
    mu = 3.0
    R = _random_rotations(rng, len(tets))
    K = oracle.stiffness_matrix(tets, Dm_inv, vol, mu, n).toarray()
    b = oracle.projection_rhs(R, tets, Dm_inv, vol, mu, n)
    x = X + 0.1 * rng.normal(size=X.shape)
    d = rng.normal(size=X.shape)
    f = oracle.elastic_forces(x, R, tets, Dm_inv, vol, mu)
    e0 = oracle.pd_energy(x, R, tets, Dm_inv, vol, mu)
    e1 = oracle.pd_energy(x + d, R, tets, Dm_inv, vol, mu)
    quad = 0.5 * sum(d[:, v] @ K @ d[:, v] for v in range(3))
    assert abs((e1 - e0) - (-np.sum(f * d) + quad)) <= 1e-9 * max(1.0, abs(e1))
    np.testing.assert_allclose(f, b - K @ x, rtol=0, atol=1e-10)
    assert np.allclose(K, K.T)
    np.testing.assert_allclose(K @ np.ones(n), 0.0, atol=1e-10)   # translations cost nothing


def test_hessian_is_block_diagonal_per_coordinate():
    # Section 2.2: no x-y-z cross terms and three identical blocks
    X, tets = _small_mesh(2)
    Dm_inv, vol = oracle.element_precompute(X, tets)
    n = len(X)
    R = _random_rotations(_rng(6), len(tets))
    K = oracle.stiffness_matrix(tets, Dm_inv, vol, 2.0, n).toarray()
    x0 = X.copy()
    f0 = oracle.elastic_forces(x0, R, tets, Dm_inv, vol, 2.0)
    H = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for v in range(3):
            x = x0.copy()
            x[i, v] += 1.0
            H[:, 3 * i + v] = -(oracle.elastic_forces(x, R, tets, Dm_inv, vol, 2.0) - f0).ravel()
    np.testing.assert_allclose(H, np.kron(K, np.eye(3)), atol=1e-10)


def test_rigid_motion_is_free():
    X, tets = _small_mesh(3)
    Dm_inv, vol = oracle.element_precompute(X, tets)
    Q = _random_rotations(_rng(7), 1)[0]
    x = X @ Q.T + np.array([1.0, -2.0, 0.5])
    R = oracle.polar_rotations(oracle.deformation_gradients(x, tets, Dm_inv))
    np.testing.assert_allclose(R, np.broadcast_to(Q, R.shape), atol=1e-12)
    f = oracle.elastic_forces(x, R, tets, Dm_inv, vol, 1e4)
    assert np.abs(f).max() < 1e-8
    assert oracle.pd_energy(x, R, tets, Dm_inv, vol, 1e4) < 1e-20


def test_contact_force_is_minus_gradient():
    X, tets = _small_mesh(4)
    rng = _rng(8)
    k = 5
    nodes = rng.integers(0, len(X), size=(k, 4)).astype(np.int32)
    nodes[0, 2:] = -1
    w = rng.uniform(size=(k, 4))
    w[0, 2:] = 0.0
    w /= w.sum(1, keepdims=True)
    c = scenes.Contacts(nodes, w, rng.normal(size=(k, 3)), rng.uniform(1, 5, size=k))
    x = X + 0.1 * rng.normal(size=X.shape)
    f = oracle.contact_forces(c, x)
    d = rng.normal(size=X.shape)
    eps = 1e-4
    fd = -(oracle.contact_energy(c, x + eps * d) - oracle.contact_energy(c, x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(f * d)) < 1e-8 * max(1, abs(fd))


# ---------------------------------------------------------------- global step
def test_one_tet_global_step_closed_form():
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tets = np.array([[0, 1, 2, 3]])
    Dm_inv, vol = oracle.element_precompute(X, tets)
    R = np.eye(3)[None]
    for a, expect in _read_gold("one_tet_closed_form.txt"):
        mu, c, t, x0 = a[0], a[1], a[2:5], a[5:8]
        K = oracle.stiffness_matrix(tets, Dm_inv, vol, mu, 4)
        b = oracle.projection_rhs(R, tets, Dm_inv, vol, mu, 4)
        con = scenes.Contacts(np.array([[3, -1, -1, -1]], np.int32), np.array([[1.0, 0, 0, 0]]),
                              t[None], np.array([c]))
        C = oracle.contact_matrix(con, 4)
        Ct = np.zeros((4, 3))
        Ct[3] = c * t
        xfix = np.array([x0, X[1], X[2]])
        x3 = oracle.global_solve(K, b, np.array([3]), np.array([0, 1, 2]), xfix, C=C, Ct=Ct)
        np.testing.assert_allclose(x3[0], expect, atol=1e-13)


def test_global_step_is_force_equilibrium():
    s = scenes.tiny_cube(2, 2, 3)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, 1e4)
    rng = _rng(9)
    x = s.X + 0.1 * rng.normal(size=s.X.shape)
    x[s.dirichlet] = s.X[s.dirichlet]
    R = _random_rotations(rng, s.E)
    con = s.contacts(0, x + np.array([0, 0, 0.5]))
    assert con.k > 0
    xs = o.full_solve(x, R, con)
    f = oracle.elastic_forces(xs, R, o.tets, o.Dm_inv, o.vol, o.mu) + oracle.contact_forces(con, xs)
    scale = np.abs(oracle.elastic_forces(x, R, o.tets, o.Dm_inv, o.vol, o.mu)).max()
    assert np.abs(f[o.part.free]).max() <= 1e-9 * scale
    np.testing.assert_array_equal(xs[s.dirichlet], x[s.dirichlet])


def test_schur_additive_update():
    # Sigma(K + C22) = Sigma(K) + C22 when C touches x_2 only (Section 3.3)
    s = scenes.tiny_cube(3, 3, 3)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, 1e4)
    p = o.part
    con = s.contacts(0, s.X + np.array([0, 0, 0.6]))
    assert con.k > 1
    C = oracle.contact_matrix(con, s.n)
    S0 = oracle.schur_complement(o.K, p.x1, p.region)
    S1 = oracle.schur_complement(o.K + C, p.x1, p.region)
    C22 = C.toarray()[np.ix_(p.region, p.region)]
    np.testing.assert_allclose(S1, S0 + C22, rtol=0, atol=1e-9 * np.abs(S0).max())
    # and Sigma equals the dense elimination of x_1 done by hand
    Kd = o.K.toarray()
    A11 = Kd[np.ix_(p.x1, p.x1)]
    A12 = Kd[np.ix_(p.x1, p.region)]
    L1 = np.linalg.cholesky(A11)
    L21t = np.linalg.solve(L1, A12)            # L_1^-1 A_12 (Eq. 9)
    S_hand = Kd[np.ix_(p.region, p.region)] - L21t.T @ L21t
    np.testing.assert_allclose(S0, S_hand, rtol=0, atol=1e-9 * np.abs(S0).max())


def _dense_algorithm1(s, outer, inner, contacts_fn, x0):
    """Algorithm 1 written out literally with dense matrices (test-local)."""
    X, tets = s.X, s.tets.astype(np.int64)
    Dm_inv, vol = oracle.element_precompute(X, tets)
    n = len(X)
    mu = s.mu
    p = oracle.Partition(n, tets, s.dirichlet, s.region)
    G = oracle.shape_gradients(Dm_inv)
    Ke = 2 * mu * vol[:, None, None] * np.einsum("eai,ebi->eab", G, G)

    def assemble(elems):
        K = np.zeros((n, n))
        for e in elems:
            K[np.ix_(tets[e], tets[e])] += Ke[e]
        return K

    Ka, Kb = assemble(p.alpha), assemble(p.beta)
    i1, i2, iD = p.x1, p.region, p.dirichlet
    A11, A12, A21 = Ka[np.ix_(i1, i1)], Ka[np.ix_(i1, i2)], Ka[np.ix_(i2, i1)]
    A22a, A22b = Ka[np.ix_(i2, i2)], Kb[np.ix_(i2, i2)]
    L1 = np.linalg.cholesky(A11)                      # preliminary partial factorisation
    L21 = np.linalg.solve(L1, A12).T                  # A_21 L_1^-T
    Sig_a = A22a - L21 @ L21.T
    x = x0.copy()

    def forces(x, R, elems):
        return oracle.elastic_forces(x, R, tets[elems], Dm_inv[elems], vol[elems], mu, n)

    for _ in range(outer):
        Ra = oracle.polar_rotations(oracle.deformation_gradients(x, tets[p.alpha], Dm_inv[p.alpha]))
        fa = forces(x, Ra, p.alpha)                                         # step 2
        y1 = np.linalg.solve(L1, fa[i1])                                    # step 3
        ft2 = fa[i2] - L21 @ y1                                             # 3.1 / 3.2
        U2 = np.zeros((len(i2), 3))
        for _ in range(inner):
            con = contacts_fn(x)                                            # 4.1
            Rb = oracle.polar_rotations(oracle.deformation_gradients(x, tets[p.beta], Dm_inv[p.beta]))
            C22 = oracle.contact_matrix(con, n).toarray()[np.ix_(i2, i2)] if con.k else 0.0
            H = Sig_a + A22b + C22                                          # 4.3
            g = ft2 + forces(x, Rb, p.beta)[i2]                             # 4.4
            if con.k:
                g = g + oracle.contact_forces(con, x)[i2]
            u2 = np.linalg.solve(H, g)                                      # 4.5
            x[i2] += u2                                                     # 4.6
            ft2 = ft2 - Sig_a @ u2                                          # 4.7
            U2 += u2
        u1 = np.linalg.solve(L1.T, y1 - L21.T @ U2)                         # 5 (full Step 3)
        x[i1] += u1
    return x


@pytest.mark.parametrize("inner", [1, 3])
def test_oracle_equals_literal_algorithm1(inner):
    s = scenes.tiny_cube(3, 3, 3)
    rng = _rng(10)
    x0 = s.X.copy()
    x0[s.region] += 0.05 * rng.normal(size=(s.m, 3))
    x0[s.dirichlet] = s.X[s.dirichlet] + np.array([0.1, 0.0, -0.05])

    def contacts_fn(x):
        return scenes.sphere_contacts(s.proxies, x, np.array([1.5, 1.5, 3.7]), 1.0, 1e6)

    assert contacts_fn(x0).k > 0
    xl = _dense_algorithm1(s, 3, inner, contacts_fn, x0)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = x0.copy()
    xo = o.step(3, inner, contacts_fn)
    np.testing.assert_allclose(xo, xl, rtol=0, atol=1e-11 * np.abs(x0).max())


def test_energy_never_increases_across_local_and_global_steps():
    s = scenes.config1(pre_indent=0.6, nx=3, ny=3, nz=6)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    rng = _rng(11)
    x = s.X.copy()
    x[o.part.free] += 0.15 * rng.normal(size=(len(o.part.free), 3))
    con = s.contacts(0, x)
    assert con.k > 0
    all_e = np.arange(s.E)
    R = o.rotations(x, all_e)
    last = o.energy(x, R, con)
    for _ in range(6):
        R = o.rotations(x, all_e)                 # local step
        e = o.energy(x, R, con)
        assert e <= last * (1 + 1e-12)
        last = e
        x = o.full_solve(x, R, con)               # global step
        e = o.energy(x, R, con)
        assert e <= last * (1 + 1e-12)
        last = e


def test_backward_euler_rest_state_stays_at_rest():
    s = scenes.config1(nx=2, ny=2, nz=4)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu, s.density, s.dt)
    o.step(3, 2, None, s.dirichlet_positions(0))
    np.testing.assert_allclose(o.x, s.X, atol=1e-12)
    np.testing.assert_allclose(o.v, 0.0, atol=1e-10)


def _read_gold_tagged(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, rest = line.split(None, 1)
        a, b = rest.split("|")
        rows.setdefault(tag, []).append((np.array(a.split(), float), np.array(b.split(), float)))
    return rows


def _be_one_tet(v0, t):
    """The one-tet backward-Euler scene of be_one_tet_closed_form.txt."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tets = np.array([[0, 1, 2, 3]])
    o = oracle.OracleSolver(X, tets, [0, 1, 2], [3], 300.0, density=24.0, dt=0.1)
    o.v[3] = v0
    con = scenes.Contacts(np.array([[3, -1, -1, -1]], np.int32), np.array([[1.0, 0, 0, 0]]),
                          np.asarray(t, float)[None], np.array([200.0]))
    return o, X, (lambda x: con)


def test_backward_euler_inertia_closed_form():
    # the inertia term m/(2 dt^2)||x - y||^2 with y = x_n + dt v_n, and
    # v_{n+1} = (x_{n+1} - x_n)/dt, against the hand solution of one tet
    gold = _read_gold_tagged("be_one_tet_closed_form.txt")
    for a, expect in gold["single"]:
        o, X, fn = _be_one_tet(a[0:3], a[3:6])
        o.step(1, 1, fn, X[:3])
        np.testing.assert_allclose(o.x[3], expect[0:3], rtol=0, atol=1e-12)
        np.testing.assert_allclose(o.v[3], expect[3:6], rtol=0, atol=1e-10)
        np.testing.assert_array_equal(o.x[:3], X[:3])
    # several steps along the axis, each with 2 outer x 2 inner iterations:
    # y must stay the start-of-step inertia target across all of them
    o, X, fn = _be_one_tet([0.0, 0.0, 3.0], [0.0, 0.0, 0.8])
    for a, expect in gold["axis"]:
        o.step(2, 2, fn, X[:3])
        np.testing.assert_allclose(o.x[3], [0.0, 0.0, expect[0]], rtol=0, atol=1e-12)
        np.testing.assert_allclose(o.v[3], [0.0, 0.0, expect[1]], rtol=0, atol=1e-10)


def test_paper_dense_flop_estimate_reading():
    # Section 3.3 quotes ~8/3 GFLOP for a Cholesky at m = 2000: that is m^3 / 3
    m = 2000
    assert abs(m ** 3 / 3 / 1e9 - 8.0 / 3.0) < 1e-12


def test_two_sided_spring_force_and_closed_form():
    # an 8-slot spring on x_a - x_b: forces are equal and opposite, and a lone
    # pair of free nodes ends at the target separation (Sherman-Morrison form)
    X, tets = _small_mesh(5)
    rng_ = _rng(12)
    x = X + 0.1 * rng_.normal(size=X.shape)
    nodes = np.full((1, 8), -1, np.int32)
    w = np.zeros((1, 8))
    nodes[0, 0], nodes[0, 4] = 3, 7
    w[0, 0], w[0, 4] = 1.0, -1.0
    t = np.array([[0.3, -0.2, 0.5]])
    c = scenes.Contacts(nodes, w, t, np.array([5.0]))
    f = oracle.contact_forces(c, x)
    np.testing.assert_allclose(f[3], -f[7], atol=1e-14)
    np.testing.assert_allclose(f[3], -5.0 * ((x[3] - x[7]) - t[0]), atol=1e-13)
    d = rng_.normal(size=x.shape)
    eps = 1e-4
    fd = -(oracle.contact_energy(c, x + eps * d) - oracle.contact_energy(c, x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(f * d)) < 1e-8 * max(1, abs(fd))
