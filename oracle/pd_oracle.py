"""Plain FP64 reference for the method of "Optimized Processing of Localized
Collisions in Projective Dynamics" (Wang et al., SCA 2020).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Written with numpy and
scipy in float64, with no blocking, fusion or reordering beyond what the paper
states, so that each function can be read against the section it cites.

Where the paper is silent or garbled, these readings are taken:
  * lambda is accepted and ignored: the energy is mu*||F - R||^2 only (Eq. 1,
    the paper sets lambda = 0 in Section 2.2).  The lambda term
    (lambda/2) tr^2(S - I) has no PD form (with R held fixed its Hessian in x
    depends on R, so the system matrix would change at every local step).
    Its PD counterpart is available as a separate volume term
    kappa ||F - T||^2, T the matrix nearest F with det T in [det_min,
    det_max]; with det_min = det_max = 1 it agrees with the lambda term to
    second order in the strain when kappa = 3 lambda / 2.  T comes from the
    principal branch of the stationarity condition (see _volume_root): the
    nearest such matrix for every contraction and inversion and for
    expansions up to about 1.9x in every direction, beyond which a matrix
    with one collapsed direction is nearer and is not taken.
  * The collision force is -W^T C (W x - t) (it follows from E_col in Eq. 7;
    the printed total force in Section 3.1 has "+ t", a sign typo).
  * The collision-prone nodes x_2 are given; E_beta is the set of tets whose
    four vertices all lie in x_2 (so that beta touches only x_2, Section 3.4).
  * Step 5 of Algorithm 1 is the full backward substitution of Step 3 in
    Section 3.2: u_1 = L_1^-T (y_1 - L_1^-1 A_12 U_2), with U_2 the sum of the
    inner-loop corrections.
  * Local step on inverted elements: R = U diag(1, 1, det(U V^T)) V^T with the
    singular values in descending order (the closest rotation in SO(3)).
  * Backward Euler (Section 2.2 says it carries over but does not show it):
    lumped mass m_i = rho * sum_{e ni i} Vol_e / 4, inertia target
    y = x_n + dt * v_n, v_{n+1} = (x_{n+1} - x_n) / dt for every node with
    x_n the positions at the end of the previous step (a prescribed node gets
    the velocity of its prescribed motion), no gravity; the x_1
    inertia belongs to the alpha part, the x_2 inertia to the beta part.
  * Dirichlet nodes are eliminated; their prescribed positions enter the
    right-hand side only.
  * Bi-phasic strain limiting (Section 5): the open set S of matrices with
    singular values strictly between sigma_min and sigma_max is taken with
    its closure, so the minimiser exists; it is Q = U clamp(Sigma) V^T from
    the SVD with non-negative singular values (an inverted F keeps its
    reflection in Q).  The mu' term is present for every element, so the
    system matrix carries mu + mu' and the target of element e is
    (mu R_e + mu' Q_e) / (mu + mu').

Parity status: every function below is pinned by tests against closed forms,
invariants, finite differences or brute force, except the multi-step
trajectory, which the paper gives no numbers for ("parity unpinned" beyond the
per-step pins).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "element_precompute", "shape_gradients", "deformation_gradients",
    "polar_rotations", "strain_limit_projection", "signed_svd", "volume_projection", "biphasic_energy", "pd_energy", "elastic_forces", "stiffness_matrix",
    "lumped_mass", "projection_rhs", "contact_matrix", "contact_forces",
    "contact_energy", "Partition", "partition", "global_solve",
    "OracleSolver", "schur_complement",
]

# The constant 4x3 matrix that maps tet vertex positions (as a 3x4 matrix
# [x0 x1 x2 x3]) to the edge matrix Ds = [x1-x0, x2-x0, x3-x0].
_S = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def element_precompute(X, tets):
    """Rest shape data of linear tets (Section 2.2, linear elements).

    Dm = [X1-X0, X2-X0, X3-X0]; Vol = |det Dm| / 6.  Returns (Dm_inv [E,3,3],
    vol [E]).  Raises ValueError on a degenerate tet."""
    P = X[tets]                               # [E, 4, 3]
    Dm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    det = np.linalg.det(Dm)
    if np.any(np.abs(det) <= 1e-300) or not np.all(np.isfinite(det)):
        raise ValueError("degenerate rest tet")
    return np.linalg.inv(Dm), np.abs(det) / 6.0


def shape_gradients(Dm_inv):
    """G_e = S Dm^-1 (4x3): F_e = [x0 x1 x2 x3] G_e."""
    return np.einsum("ab,ebc->eac", _S, Dm_inv)


def deformation_gradients(x, tets, Dm_inv):
    """F_e = Ds Dm^-1 (Section 2.2)."""
    P = x[tets]
    Ds = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    return Ds @ Dm_inv


def polar_rotations(F):
    """Local step (Section 2.2): the rotation minimising ||F - R||_F over SO(3),
    R = U V^T from the SVD F = U Sigma V^T (orthogonal Procrustes), with the
    smallest singular direction negated when det(U V^T) < 0."""
    U, s, Vt = np.linalg.svd(F)
    d = np.sign(np.linalg.det(U @ Vt))
    d[d == 0] = 1.0
    D = np.ones(F.shape[:-2] + (3,))
    D[..., 2] = d
    return (U * D[..., None, :]) @ Vt


def strain_limit_projection(F, sigma_min, sigma_max):
    """Local step of the bi-phasic term (Section 5): the matrix with singular
    values in [sigma_min, sigma_max] closest to F in the Frobenius norm,
    Q = U clamp(Sigma, sigma_min, sigma_max) V^T from the SVD F = U Sigma V^T."""
    U, s, Vt = np.linalg.svd(F)
    return (U * np.clip(s, sigma_min, sigma_max)[..., None, :]) @ Vt


def signed_svd(F):
    """F = U diag(s) V^T with U, V rotations and s = (s1, s2, s3), s1 >= s2 >=
    |s3|: the plain SVD with the smallest singular value negated when
    det F < 0 (so that s3 < 0 marks an inverted element)."""
    U, s, Vt = np.linalg.svd(F)
    du = np.where(np.linalg.det(U) < 0, -1.0, 1.0)
    dv = np.where(np.linalg.det(Vt) < 0, -1.0, 1.0)
    U, s, Vt = U.copy(), s.copy(), Vt.copy()
    U[..., :, 2] *= du[..., None]       # third columns of U and V flipped
    Vt[..., 2, :] *= dv[..., None]      # into rotations, the sign moved to s_3
    s[..., 2] *= du * dv
    return U, s, Vt


def _volume_root(sig, v):
    """The diagonal tau nearest sig with prod(tau) = v > 0 on the principal
    branch of the stationarity condition (tau_i - s_i) tau_i = -c, i.e.
    tau_i(c) = (s_i + sqrt(s_i^2 - 4c)) / 2, each decreasing in c, for
    c <= min_i s_i^2 / 4.  prod(tau(c)) = v is solved for c by bisection to
    the resolution of float64.  When even the branch end c = min s_i^2 / 4
    leaves prod(tau) > v (an element stretched about twofold or more in
    every direction), the branch end is returned."""
    sig = np.asarray(sig, dtype=np.float64)

    def tau(c):
        r = np.sqrt(np.maximum(sig * sig - 4.0 * c, 0.0))
        # the form without cancellation: for s_i < 0, tau_i = 2c / (s_i - r)
        with np.errstate(divide="ignore", invalid="ignore"):
            neg = np.where(sig - r != 0.0, 2.0 * c / (sig - r), 0.0)
        return np.where(sig >= 0.0, 0.5 * (sig + r), neg)

    p0 = float(np.prod(sig))
    if p0 < v:                           # contraction or inversion: c < 0
        hi = 0.0
        lo = -max(1.0, float(np.max(sig * sig)))
        while np.prod(tau(lo)) < v:
            lo *= 4.0
    else:                                # expansion: 0 < c <= min s_i^2 / 4
        lo = 0.0
        hi = float(np.min(sig * sig)) / 4.0
        if np.prod(tau(hi)) > v:
            return tau(hi)
    # invariant: prod(tau(lo)) >= v >= prod(tau(hi))
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if np.prod(tau(mid)) >= v:
            lo = mid
        else:
            hi = mid
    a, b = tau(lo), tau(hi)
    return a if abs(np.prod(a) - v) <= abs(np.prod(b) - v) else b


def volume_projection(F, det_min, det_max):
    """Local step of the PD volume term kappa ||F - T||^2 (the PD form of
    the lambda term of Eq. 1): T is the matrix nearest F whose determinant
    lies in [det_min, det_max] (0 < det_min <= det_max).  From the signed
    SVD F = U diag(s) V^T, T = U diag(tau) V^T with tau the diagonal nearest
    s whose product is the bound that det F violates (T = F inside the
    bounds); see _volume_root."""
    F = np.asarray(F, dtype=np.float64)
    flat = F.reshape(-1, 3, 3)
    out = flat.copy()
    U, s, Vt = signed_svd(flat)
    for e in range(len(flat)):
        d = float(np.prod(s[e]))
        if det_min <= d <= det_max:
            continue
        t = _volume_root(s[e], det_min if d < det_min else det_max)
        out[e] = (U[e] * t[None, :]) @ Vt[e]
    return out.reshape(F.shape)


def biphasic_energy(x, R, Q, tets, Dm_inv, vol, mu, mu_prime):
    """E_hat'(x, R, Q) = sum_e Vol_e (mu' ||F_e - Q_e||^2 + mu ||F_e - R_e||^2)
    (Section 5)."""
    F = deformation_gradients(x, tets, Dm_inv)
    return float(np.sum(vol * (mu_prime * np.sum((F - Q) ** 2, axis=(1, 2))
                               + mu * np.sum((F - R) ** 2, axis=(1, 2)))))


def pd_energy(x, R, tets, Dm_inv, vol, mu, elems=None):
    """E_hat(x, R) = sum_e Vol_e * mu * ||F_e(x) - R_e||_F^2 (Eqs. 2-3)."""
    if elems is not None:
        tets, Dm_inv, vol, R = tets[elems], Dm_inv[elems], vol[elems], R[elems] if len(R) != len(elems) else R
    F = deformation_gradients(x, tets, Dm_inv)
    return float(np.sum(vol * mu * np.sum((F - R) ** 2, axis=(1, 2))))


def elastic_forces(x, R, tets, Dm_inv, vol, mu, n=None):
    """f = -dE_hat/dx with R fixed (Section 2.2): P = 2 mu (F - R) and
    f_e = -Vol_e P G_e^T, scattered to the four vertices.  Returns [n, 3]."""
    n = len(x) if n is None else n
    F = deformation_gradients(x, tets, Dm_inv)
    P = 2.0 * mu * (F - R)
    G = shape_gradients(Dm_inv)
    fe = -vol[:, None, None] * np.einsum("eij,eaj->eai", P, G)   # [E, 4, 3]
    f = np.zeros((n, 3))
    for a in range(4):
        np.add.at(f, tets[:, a], fe[:, a])
    return f


def stiffness_matrix(tets, Dm_inv, vol, mu, n):
    """Scalar PD matrix K = sum_e 2 mu Vol_e G_e G_e^T (n x n); the 3n x 3n
    Hessian of E_hat is K (x) I_3 (Section 2.2, block-diagonal per coordinate)."""
    G = shape_gradients(Dm_inv)
    Ke = 2.0 * mu * vol[:, None, None] * np.einsum("eai,ebi->eab", G, G)
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))


def lumped_mass(tets, vol, density, n):
    """m_i = density * sum over incident tets of Vol_e / 4 (backward Euler)."""
    m = np.zeros(n)
    for a in range(4):
        np.add.at(m, tets[:, a], density * vol / 4.0)
    return m


def projection_rhs(R, tets, Dm_inv, vol, mu, n):
    """b = sum_e 2 mu Vol_e G_e R_e^T scattered, so that E_hat(x) for fixed R
    equals sum_v (1/2 x_v^T K x_v - b_v^T x_v) + const.  Returns [n, 3]."""
    G = shape_gradients(Dm_inv)
    be = 2.0 * mu * vol[:, None, None] * np.einsum("eaj,eij->eai", G, R)   # [E, 4, 3]
    b = np.zeros((n, 3))
    for a in range(4):
        np.add.at(b, tets[:, a], be[:, a])
    return b


def _contact_W(contacts, n):
    k = contacts.k
    rows = np.repeat(np.arange(k), contacts.nodes.shape[1])
    cols = contacts.nodes.ravel()
    vals = contacts.w.ravel()
    keep = cols >= 0
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(k, n))


def contact_matrix(contacts, n):
    """C_22 = W^T C W over all nodes (Eq. 8), C = diag(c_j) of active springs."""
    W = _contact_W(contacts, n)
    return (W.T @ sp.diags(contacts.stiffness) @ W).tocsr()


def contact_forces(contacts, x):
    """f_col = -W^T C (W x - t) (Section 3.1, sign as derived from Eq. 7)."""
    W = _contact_W(contacts, len(x))
    r = W @ x - contacts.target
    return -(W.T @ (contacts.stiffness[:, None] * r))


def contact_energy(contacts, x):
    """E_col = sum_j c_j / 2 ||p_j - t_j||^2 over active springs (Section 2.3)."""
    W = _contact_W(contacts, len(x))
    r = W @ x - contacts.target
    return float(0.5 * np.sum(contacts.stiffness[:, None] * r * r))


class Partition:
    """Node and element split of Section 3.4 / Figure 2."""

    def __init__(self, n, tets, dirichlet, region):
        self.n = n
        self.dirichlet = np.asarray(dirichlet, dtype=np.int64)
        self.region = np.asarray(region, dtype=np.int64)
        is_d = np.zeros(n, bool)
        is_d[self.dirichlet] = True
        is_r = np.zeros(n, bool)
        is_r[self.region] = True
        if np.any(is_d & is_r):
            raise ValueError("region and Dirichlet sets overlap")
        self.free = np.nonzero(~is_d)[0]
        self.x1 = np.nonzero(~is_d & ~is_r)[0]
        self.beta = np.nonzero(is_r[tets].all(axis=1))[0]
        self.alpha = np.nonzero(~is_r[tets].all(axis=1))[0]


def partition(n, tets, dirichlet, region):
    return Partition(n, tets, dirichlet, region)


def global_solve(K, b, free, fixed, x_fixed, extra_diag=None, extra_rhs=None, C=None, Ct=None):
    """Minimise the quadratic sum_v 1/2 x_v^T (K + C) x_v - rhs_v^T x_v over the
    free nodes with the fixed nodes held at x_fixed (the PD global step,
    Section 2.2, with the penalty terms of Section 2.3 folded in).
    K: n x n sparse; b: [n, 3]; C: optional n x n sparse contact matrix with
    Ct = W^T C t [n, 3]; extra_diag / extra_rhs: inertia terms.  Solves the
    free block directly (sparse LU, all three coordinates at once)."""
    M = K if C is None else (K + C)
    rhs = b.copy()
    if Ct is not None:
        rhs = rhs + Ct
    if extra_diag is not None:
        M = M + sp.diags(extra_diag)
        rhs = rhs + extra_rhs
    M = M.tocsr()
    Mff = M[free][:, free].tocsc()
    r = rhs[free] - M[free][:, fixed] @ x_fixed
    lu = spla.splu(Mff, permc_spec="MMD_AT_PLUS_A")
    return lu.solve(r)


def schur_complement(A, idx1, idx2):
    """Sigma = A_22 - A_21 A_11^-1 A_12 (Eq. 10), dense, from a sparse A."""
    A = A.tocsr()
    A11 = A[idx1][:, idx1].tocsc()
    A12 = A[idx1][:, idx2].toarray()
    A22 = A[idx2][:, idx2].toarray()
    Z = spla.splu(A11, permc_spec="MMD_AT_PLUS_A").solve(A12)
    return A22 - A12.T @ Z


class OracleSolver:
    """Algorithm 1 (Section 3.4), computed without the Schur split.

    Each inner iteration solves the full free-node system with R_alpha from the
    start of the outer iteration, R_beta and the contacts of this inner
    iteration, and keeps only x_2 from that solve; x_1 is taken from the last
    such solve when the inner loop ends.  This equals the Schur-complement
    form because minimising over x_1 first leaves the reduced energy
    E~_alpha(x_2) the paper's inner loop descends (Eq. 12)."""

    def __init__(self, X, tets, dirichlet, region, mu, density=0.0, dt=0.0, mu_prime=0.0,
                 sigma_min=0.0, sigma_max=np.inf, kappa=0.0, det_min=1.0, det_max=1.0):
        self.X = np.asarray(X, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.n = len(X)
        self.mu = float(mu)
        self.dt = float(dt)
        # bi-phasic strain limiting (Section 5); mu_prime = 0 turns it off
        self.mu_prime = float(mu_prime)
        self.sigma = (float(sigma_min), float(sigma_max))
        # PD volume term kappa ||F - T||^2 (the lambda term of Eq. 1 in PD
        # form); kappa = 0 turns it off
        self.kappa = float(kappa)
        self.det = (float(det_min), float(det_max))
        self.Dm_inv, self.vol = element_precompute(self.X, self.tets)
        self.part = Partition(self.n, self.tets, dirichlet, region)
        self.K = stiffness_matrix(self.tets, self.Dm_inv, self.vol, self.mu + self.mu_prime + self.kappa, self.n)
        self.mass = lumped_mass(self.tets, self.vol, density, self.n) if dt > 0 else None
        self.x = self.X.copy()
        self.v = np.zeros_like(self.X)
        self.stats = {"solves": 0}

    def set_dirichlet(self, pos):
        self.x[self.part.dirichlet] = pos

    def rotations(self, x, elems):
        F = deformation_gradients(x, self.tets[elems], self.Dm_inv[elems])
        return polar_rotations(F)

    def projections(self, x, elems):
        """Q_e of the bi-phasic term (Section 5) for the given elements."""
        F = deformation_gradients(x, self.tets[elems], self.Dm_inv[elems])
        return strain_limit_projection(F, *self.sigma)

    def volume_targets(self, x, elems):
        """T_e of the volume term for the given elements."""
        F = deformation_gradients(x, self.tets[elems], self.Dm_inv[elems])
        return volume_projection(F, *self.det)

    def full_solve(self, x, R, contacts, y=None, Q=None, T=None):
        """Argmin over free x of E_hat(x; R) (with the bi-phasic term at Q and
        the volume term at T when present) + E_col (+ inertia), Dirichlet
        fixed."""
        b = projection_rhs(R, self.tets, self.Dm_inv, self.vol, self.mu, self.n)
        if self.mu_prime > 0:
            b = b + projection_rhs(Q, self.tets, self.Dm_inv, self.vol, self.mu_prime, self.n)
        if self.kappa > 0:
            b = b + projection_rhs(T, self.tets, self.Dm_inv, self.vol, self.kappa, self.n)
        C = Ct = None
        if contacts is not None and contacts.k > 0:
            C = contact_matrix(contacts, self.n)
            W = _contact_W(contacts, self.n)
            Ct = W.T @ (contacts.stiffness[:, None] * contacts.target)
        ed = er = None
        if self.mass is not None:
            ed = self.mass / self.dt ** 2
            er = ed[:, None] * y
        p = self.part
        xf = global_solve(self.K, b, p.free, p.dirichlet, x[p.dirichlet], ed, er, C, Ct)
        out = x.copy()
        out[p.free] = xf
        self.stats["solves"] += 1
        return out

    def step(self, outer_iters, inner_iters, contacts_fn=None, dirichlet_pos=None):
        """One time step (quasistatic if dt == 0): Algorithm 1 repeated
        outer_iters times.  contacts_fn(x) -> Contacts is called once per inner
        iteration with the current x_2 (the detection step 4.1)."""
        p = self.part
        x_n = self.x.copy()       # positions at the end of the previous step
        if dirichlet_pos is not None:
            self.set_dirichlet(dirichlet_pos)
        y = (x_n + self.dt * self.v) if self.mass is not None else None
        R = np.zeros((len(self.tets), 3, 3))
        Q = np.zeros((len(self.tets), 3, 3)) if self.mu_prime > 0 else None
        T = np.zeros((len(self.tets), 3, 3)) if self.kappa > 0 else None
        for _ in range(outer_iters):
            R[p.alpha] = self.rotations(self.x, p.alpha)          # step 1
            if Q is not None:
                Q[p.alpha] = self.projections(self.x, p.alpha)
            if T is not None:
                T[p.alpha] = self.volume_targets(self.x, p.alpha)
            virt = None
            for _ in range(inner_iters):
                contacts = contacts_fn(self.x) if contacts_fn is not None else None   # 4.1
                R[p.beta] = self.rotations(self.x, p.beta)        # 4.2
                if Q is not None:
                    Q[p.beta] = self.projections(self.x, p.beta)
                if T is not None:
                    T[p.beta] = self.volume_targets(self.x, p.beta)
                virt = self.full_solve(self.x, R, contacts, y, Q, T)  # 4.3-4.5
                self.x[p.region] = virt[p.region]                 # 4.6
            self.x[p.x1] = virt[p.x1]                             # 5
        if self.mass is not None:
            self.v = (self.x - x_n) / self.dt
        return self.x

    def energy(self, x, R, contacts=None, y=None, Q=None, T=None):
        """E_hat (or E_hat' with Q, plus the volume term with T) + E_col
        (+ inertia) at x for fixed R, Q, T and contacts."""
        if self.mu_prime > 0:
            e = biphasic_energy(x, R, Q, self.tets, self.Dm_inv, self.vol, self.mu, self.mu_prime)
        else:
            e = pd_energy(x, R, self.tets, self.Dm_inv, self.vol, self.mu)
        if self.kappa > 0:
            F = deformation_gradients(x, self.tets, self.Dm_inv)
            e += float(np.sum(self.vol * self.kappa * np.sum((F - T) ** 2, axis=(1, 2))))
        if contacts is not None and contacts.k > 0:
            e += contact_energy(contacts, x)
        if self.mass is not None and y is not None:
            e += float(0.5 * np.sum(self.mass[:, None] / self.dt ** 2 * (x - y) ** 2))
        return e
