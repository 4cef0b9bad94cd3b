"""The benchmark scenes, as plain arrays.

Sizes follow the paper's test models (Section 5: ~0.5-0.65M tets, ~0.1M nodes,
1.5-5% collision-prone nodes).  The paper's meshes are not public, so every
scene is a seeded voxel mesh with the same size and region fraction.
"""
from dataclasses import dataclass, field
from typing import Callable, Optional
import math
import numpy as np

from .mesh import voxel_mesh, grid_mesh, boundary_nodes, boundary_faces_outward, jitter_interior, node_adjacency


@dataclass
class Contacts:
    """Active penalty springs: proxy j sits at sum_a w[j,a] * x[nodes[j,a]]."""
    nodes: np.ndarray      # [k, 4] int32, -1 pads unused slots
    w: np.ndarray          # [k, 4] float64
    target: np.ndarray     # [k, 3] float64
    stiffness: np.ndarray  # [k] float64

    @property
    def k(self):
        return int(self.nodes.shape[0])


def empty_contacts():
    return Contacts(np.zeros((0, 4), np.int32), np.zeros((0, 4)), np.zeros((0, 3)), np.zeros(0))


def _node_contacts(nodes, target, stiffness):
    k = len(nodes)
    n4 = np.full((k, 4), -1, dtype=np.int32)
    n4[:, 0] = nodes
    w = np.zeros((k, 4))
    w[:, 0] = 1.0
    return Contacts(n4, w, np.asarray(target, dtype=np.float64).reshape(k, 3),
                    np.full(k, float(stiffness)))


def rotation_z(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rotation_x(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


@dataclass
class Scene:
    name: str
    X: np.ndarray            # [n, 3] rest positions
    tets: np.ndarray         # [E, 4] int32
    dirichlet: np.ndarray    # [nd] int32
    region: np.ndarray       # [m] int32, the collision-prone nodes x_2
    proxies: np.ndarray      # [p] int32, region nodes that carry collision proxies
    mu: float = 1e4
    lam: float = 4e4         # accepted and ignored (the paper sets lambda = 0)
    density: float = 1000.0
    dt: float = 0.0          # 0 = quasistatic
    outer_iters: int = 10
    inner_iters: int = 1
    steps: int = 5
    stiffness: float = 1e6
    dirichlet_positions: Callable[[int], np.ndarray] = None   # step -> [nd, 3]
    contacts: Callable[[int, np.ndarray], Contacts] = None    # (step, x [n,3]) -> Contacts
    info: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.X.shape[0])

    @property
    def E(self):
        return int(self.tets.shape[0])

    @property
    def m(self):
        return int(self.region.shape[0])


def sphere_contacts(proxies, x, centre, radius, stiffness):
    """Proxies inside a rigid sphere, projected to its surface."""
    p = x[proxies]
    d = p - np.asarray(centre)[None, :]
    r = np.linalg.norm(d, axis=1)
    act = r < radius
    if not np.any(act):
        return empty_contacts()
    t = np.asarray(centre)[None, :] + radius * d[act] / r[act, None]
    return _node_contacts(proxies[act], t, stiffness)


def cylinder_contacts(nodes, x, origin, axis, radius, length, stiffness):
    """Nodes inside a rigid finite cylinder, pushed radially to its surface."""
    if len(nodes) == 0:
        return empty_contacts()
    p = x[nodes] - np.asarray(origin)[None, :]
    a = np.asarray(axis) / np.linalg.norm(axis)
    s = p @ a
    radial = p - s[:, None] * a[None, :]
    r = np.linalg.norm(radial, axis=1)
    act = (r < radius) & (s > 0.0) & (s < length) & (r > 1e-12)
    if not np.any(act):
        return empty_contacts()
    t = (np.asarray(origin)[None, :] + s[act, None] * a[None, :]
         + radius * radial[act] / r[act, None])
    return _node_contacts(nodes[act], t, stiffness)


def pair_contacts(side_a, side_b, x, gap, stiffness):
    """Two-sided springs between surface nodes of opposite sides closer than
    `gap`: spring on d = x_a - x_b with frozen target gap * (x_a - x_b)/|x_a - x_b|,
    i.e. the pair is pushed apart to distance `gap` (8-slot rows: +1 on a, -1 on b)."""
    if len(side_a) == 0 or len(side_b) == 0:
        return Contacts(np.zeros((0, 8), np.int32), np.zeros((0, 8)), np.zeros((0, 3)), np.zeros(0))
    pa, pb = x[side_a], x[side_b]
    d2 = ((pa[:, None, :] - pb[None, :, :]) ** 2).sum(-1)
    j = np.argmin(d2, axis=1)
    dist = np.sqrt(d2[np.arange(len(side_a)), j])
    act = (dist < gap) & (dist > 1e-12)
    ia, ib = side_a[act], side_b[j[act]]
    k = len(ia)
    nodes = np.full((k, 8), -1, np.int32)
    w = np.zeros((k, 8))
    nodes[:, 0], nodes[:, 4] = ia, ib
    w[:, 0], w[:, 4] = 1.0, -1.0
    d = x[ia] - x[ib]
    target = gap * d / np.linalg.norm(d, axis=1, keepdims=True)
    return Contacts(nodes, w, target, np.full(k, float(stiffness)))


def _cat(*cs):
    cs = [c for c in cs if c.k > 0]
    if not cs:
        return empty_contacts()
    return Contacts(np.concatenate([c.nodes for c in cs]), np.concatenate([c.w for c in cs]),
                    np.concatenate([c.target for c in cs]), np.concatenate([c.stiffness for c in cs]))


# --------------------------------------------------------------------------
# Configuration 1: 10 x 10 x 40 cube column, sphere indenter on top.
# --------------------------------------------------------------------------
def config1(seed=0, pre_indent=0.0, nx=10, ny=10, nz=40):
    """Column of nx*ny*nz unit cubes (z up), bottom fixed, top two node layers
    collision-prone; a rigid sphere of radius 3 starts tangent to the top face
    (centre (5, 5, 43)) and descends at 0.5 per second; backward Euler with
    dt = 1/30.  `pre_indent` lowers the sphere so more proxies are active."""
    X, tets, g = grid_mesh(nx, ny, nz, 1.0)
    X = jitter_interior(X, tets, 0.1, seed)
    dirichlet = np.nonzero(g[:, 2] == 0)[0].astype(np.int32)
    region = np.nonzero(g[:, 2] >= nz - 1)[0].astype(np.int32)
    proxies = np.nonzero(g[:, 2] == nz)[0].astype(np.int32)
    dt = 1.0 / 30.0
    Xd = X[dirichlet].copy()
    cx, cy = nx / 2.0, ny / 2.0
    stiffness = 1e6

    def centre(step):
        return np.array([cx, cy, nz + 3.0 - pre_indent - 0.5 * (step + 1) * dt])

    def contacts(step, x):
        return sphere_contacts(proxies, x, centre(step), 3.0, stiffness)

    return Scene("config1", X, tets, dirichlet, region, proxies, mu=1e4, lam=4e4,
                 density=1000.0, dt=dt, outer_iters=10, inner_iters=1, steps=5,
                 stiffness=stiffness, dirichlet_positions=lambda step: Xd.copy(),
                 contacts=contacts, info={"sphere_centre": centre})


def tiny_cube(nx=2, ny=2, nz=2, seed=0):
    """A few cubes with the bottom fixed and the top layer collision-prone."""
    X, tets, g = grid_mesh(nx, ny, nz, 1.0)
    X = jitter_interior(X, tets, 0.1, seed)
    dirichlet = np.nonzero(g[:, 2] == 0)[0].astype(np.int32)
    region = np.nonzero(g[:, 2] >= nz - 1)[0].astype(np.int32)
    proxies = np.nonzero(g[:, 2] == nz)[0].astype(np.int32)
    Xd = X[dirichlet].copy()

    def contacts(step, x):
        return sphere_contacts(proxies, x, np.array([nx / 2, ny / 2, nz + 0.8]), 1.0, 1e6)

    return Scene("tiny_cube", X, tets, dirichlet, region, proxies, dt=0.0, outer_iters=3,
                 steps=1, dirichlet_positions=lambda step: Xd.copy(), contacts=contacts)


# --------------------------------------------------------------------------
# Configurations 2-3, 5: an elbow made of two cylinders joined at 90 degrees.
# --------------------------------------------------------------------------
_R, _L = 8.0, 60.0


def _elbow_inside(c):
    x, y, z = c[..., 0], c[..., 1], c[..., 2]
    cyl_a = (x >= -_L) & (x <= 0.0) & (y * y + z * z <= _R * _R)
    cyl_b = (y >= 0.0) & (y <= _L) & (x * x + z * z <= _R * _R)
    ball = x * x + y * y + z * z <= _R * _R
    return cyl_a | cyl_b | ball


def _elbow_voxels(h):
    lo = np.array([-_L - h, -_R - h, -_R - h])
    hi = np.array([_R + h, _L + h, _R + h])
    shape = np.ceil((hi - lo) / h).astype(int)
    # x = -L is a lattice plane, so cap A is one flat layer of nodes
    ii, jj, kk = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
    centres = lo[None, None, None, :] + h * (np.stack([ii, jj, kk], -1) + 0.5)
    return _elbow_inside(centres), lo


def elbow(h=0.585, seed=0, region_fraction=0.05, inner_iters=1, contact_mode="self"):
    """Elbow: cylinders A (axis (-60,0,0)->(0,0,0)) and B ((0,0,0)->(0,60,0)),
    radius 8, plus a ball of radius 8 at the joint, voxelised at spacing h
    (h = 0.585 gives ~596K tets).  Cap A is fixed; cap B is rotated about the
    z axis through the origin.  Flexion is phi(s) = 2 deg * s measured from a
    straight arm; the rest shape is phi = 90 deg.  The collision-prone region
    is the ceil(fraction * n) nodes within two layers of the surface that are
    nearest the inner crease point (-8, 8, 0)."""
    keep, lo = _elbow_voxels(h)
    X, tets, g = voxel_mesh(keep, h, lo)
    n = len(X)
    # no jitter: the voxel lattice stays regular, as the paper's embedding meshes were
    surf = boundary_nodes(tets, n)
    indptr, indices = node_adjacency(tets, n)
    depth = np.where(surf, 0, 99)
    frontier = np.nonzero(surf)[0]
    for layer in (1, 2):
        nbr = indices[np.concatenate([np.arange(indptr[i], indptr[i + 1]) for i in frontier])] if len(frontier) else []
        nbr = np.unique(nbr)
        new = nbr[depth[nbr] > layer]
        depth[new] = layer
        frontier = new
    cand = np.nonzero(depth <= 2)[0]
    pc = np.array([-_R, _R, 0.0])
    dist = np.linalg.norm(X[cand] - pc[None, :], axis=1)
    m = int(math.ceil(region_fraction * n))
    order = np.lexsort((cand, dist))
    region = np.sort(cand[order[:m]]).astype(np.int32)
    cap_a = np.nonzero(X[:, 0] < -_L + 0.5 * h)[0]
    cap_b = np.nonzero(X[:, 1] > _L - 0.5 * h)[0]
    dirichlet = np.concatenate([cap_a, cap_b]).astype(np.int32)
    in_region = np.zeros(n, bool)
    in_region[region] = True
    proxies = np.nonzero(in_region & surf)[0].astype(np.int32)
    XA = X[cap_a].copy()
    XB = X[cap_b].copy()
    stiffness = 1e6

    def theta(step):
        return math.radians(2.0 * step - 90.0)

    def dirichlet_positions(step):
        return np.concatenate([XA, XB @ rotation_z(theta(step)).T])

    # self-contact: A-side proxies against B's rigidly rotated cylinder, and
    # B-side proxies against A's cylinder, using rest-pose implicit surfaces.
    side_a = proxies[(X[proxies, 0] + X[proxies, 1]) < 0.0]
    side_b = proxies[(X[proxies, 0] + X[proxies, 1]) >= 0.0]
    # eligible only if outside the other cylinder at rest
    rb = np.sqrt(X[side_a, 0] ** 2 + X[side_a, 2] ** 2)
    side_a = side_a[(rb >= _R) | (X[side_a, 1] <= 0.0)]
    ra = np.sqrt(X[side_b, 1] ** 2 + X[side_b, 2] ** 2)
    side_b = side_b[(ra >= _R) | (X[side_b, 0] >= 0.0)]

    def contacts(step, x):
        # theta(step) is measured from the rest L-shape, where B points along +y
        axis_b = rotation_z(theta(step)) @ np.array([0.0, 1.0, 0.0])
        ca = cylinder_contacts(side_b, x, np.zeros(3), np.array([-1.0, 0.0, 0.0]), _R, _L, stiffness)
        cb = cylinder_contacts(side_a, x, np.zeros(3), axis_b, _R, _L, stiffness)
        return _cat(ca, cb)

    all_a = proxies[(X[proxies, 0] + X[proxies, 1]) < 0.0]
    all_b = proxies[(X[proxies, 0] + X[proxies, 1]) >= 0.0]
    # point-triangle self-contact (config 2): the outward surface triangles of
    # the region, split by the same plane; a side's nodes are tested against
    # the other side's triangles, skipping pairs within 3h at rest (the
    # surface that runs continuously through the crease)
    faces = boundary_faces_outward(X, tets)
    faces = faces[in_region[faces].all(axis=1)]
    fc = X[faces].mean(axis=1)
    tris_a = faces[(fc[:, 0] + fc[:, 1]) < 0.0].astype(np.int32)
    tris_b = faces[(fc[:, 0] + fc[:, 1]) >= 0.0].astype(np.int32)

    def self_pairs(x, gap=None):
        return pair_contacts(all_a, all_b, x, 2.0 * h if gap is None else gap, stiffness)

    return Scene("elbow", X, tets, dirichlet, region, proxies, mu=1e4, lam=0.0,
                 density=1000.0, dt=0.0, outer_iters=10, inner_iters=inner_iters, steps=60,
                 stiffness=stiffness, dirichlet_positions=dirichlet_positions,
                 contacts=contacts,
                 info={"h": h, "theta": theta, "rest_step": 45, "self_pairs": self_pairs,
                       "pair_sides": (all_a, all_b), "tri_sides": (all_a, tris_a, all_b, tris_b),
                       "tri_gap": h, "tri_rest_min": 3.0 * h})


def closed_pose(scene, angle=40.0, band=8.0):
    """Initial positions of an elbow with the joint closed by `angle` degrees
    beyond the rest L (flexion step 45 + angle / 2): every node turned about
    the hinge by angle * smoothstep across a band of half-width `band` around
    the plane x + y = 0 between the two segments, so no element inverts and
    the crease surfaces of the two segments meet.  Returns (x, flexion step)."""
    X = scene.X
    d = (X[:, 0] + X[:, 1]) / math.sqrt(2.0)
    t = np.clip((d + band) / (2.0 * band), 0.0, 1.0)
    ang = np.radians(angle) * t * t * (3.0 - 2.0 * t)
    c, sn = np.cos(ang), np.sin(ang)
    x = X.copy()
    x[:, 0] = c * X[:, 0] - sn * X[:, 1]
    x[:, 1] = sn * X[:, 0] + c * X[:, 1]
    return x, int(round(45 + angle / 2.0))


def small_elbow(h=2.0, seed=0, region_fraction=0.05, inner_iters=1):
    """The elbow at a coarse spacing, for parity runs the oracle finishes fast."""
    s = elbow(h=h, seed=seed, region_fraction=region_fraction, inner_iters=inner_iters)
    s.name = "small_elbow"
    return s


# --------------------------------------------------------------------------
# Configuration 4: two stacked slabs ("lips") with a hinged lower slab.
# --------------------------------------------------------------------------
def slabs(nx=120, ny=60, nz=9, gap=0.5, m=6250, seed=0):
    """Two slabs of nx*ny*nz unit cubes, the upper one `gap` above the lower.
    The upper slab's top face is fixed; the lower slab's bottom face rotates
    about its back-bottom edge (y = ny, z = 0) by 0 -> 15 degrees, closing the
    front of the gap.  The collision-prone region is the m nodes nearest the
    front half of the gap mid-plane."""
    Xl, tl, gl = grid_mesh(nx, ny, nz, 1.0, (0.0, 0.0, 0.0))
    Xu, tu, gu = grid_mesh(nx, ny, nz, 1.0, (0.0, 0.0, nz + gap))
    X = np.concatenate([Xl, Xu])
    tets = np.concatenate([tl, tu + len(Xl)]).astype(np.int32)
    n = len(X)
    lower = np.arange(n) < len(Xl)
    zmid = nz + 0.5 * gap
    # distance to the rectangle [0,nx] x [0, ny/2] on the mid-plane
    dy = np.maximum(X[:, 1] - ny / 2.0, 0.0)
    d = np.sqrt(dy ** 2 + (X[:, 2] - zmid) ** 2)
    order = np.lexsort((np.arange(n), d))
    region = np.sort(order[:m]).astype(np.int32)
    bottom = np.nonzero(lower & (np.abs(X[:, 2]) < 1e-9))[0]
    top = np.nonzero((~lower) & (np.abs(X[:, 2] - (2 * nz + gap)) < 1e-9))[0]
    dirichlet = np.concatenate([top, bottom]).astype(np.int32)
    Xt, Xb = X[top].copy(), X[bottom].copy()
    hinge = np.array([0.0, float(ny), 0.0])
    steps = 60

    def ang(step):
        return math.radians(15.0 * min(step + 1, steps) / steps)

    def dirichlet_positions(step):
        R = rotation_x(-ang(step))   # front (y = 0) of the lower slab moves up, closing the gap
        return np.concatenate([Xt, (Xb - hinge) @ R.T + hinge])

    in_region = np.zeros(n, bool)
    in_region[region] = True
    surf = boundary_nodes(tets, n)
    prox_l = np.nonzero(in_region & surf & lower & (np.abs(X[:, 2] - nz) < 1e-9))[0].astype(np.int32)
    prox_u = np.nonzero(in_region & surf & ~lower & (np.abs(X[:, 2] - (nz + gap)) < 1e-9))[0].astype(np.int32)
    proxies = np.concatenate([prox_l, prox_u]).astype(np.int32)

    def contacts(step, x):
        out = []
        zl = x[prox_l, 2]
        act = zl > zmid
        if np.any(act):
            t = x[prox_l[act]].copy()
            t[:, 2] = zmid
            out.append(_node_contacts(prox_l[act], t, 1e6))
        zu = x[prox_u, 2]
        act = zu < zmid
        if np.any(act):
            t = x[prox_u[act]].copy()
            t[:, 2] = zmid
            out.append(_node_contacts(prox_u[act], t, 1e6))
        return _cat(*out) if out else empty_contacts()

    return Scene("slabs", X, tets, dirichlet, region, proxies, mu=1e4, lam=4e4,
                 density=1000.0, dt=0.0, outer_iters=10, inner_iters=1, steps=steps,
                 stiffness=1e6, dirichlet_positions=dirichlet_positions, contacts=contacts)
