"""Voxel tetrahedral meshes: unit cubes split into five tetrahedra.

Neighbouring cubes alternate between the two mirror-image five-tet splits by
the parity of (i + j + k), so that the face diagonals of adjacent cubes agree
and the mesh is conforming.
"""
import numpy as np

# Cube corner b = dx + 2*dy + 4*dz.  Split A keeps the four corners with an
# even number of set bits as "corner tets" and puts the odd ones in the middle;
# split B is its mirror image.
_SPLIT_A = np.array([[0, 1, 2, 4],   # corner 000
                     [3, 1, 2, 7],   # corner 110
                     [5, 1, 4, 7],   # corner 101
                     [6, 2, 4, 7],   # corner 011
                     [1, 2, 4, 7]],  # middle tet
                    dtype=np.int64)
_SPLIT_B = np.array([[1, 0, 3, 5],   # corner 100
                     [2, 0, 3, 6],   # corner 010
                     [4, 0, 5, 6],   # corner 001
                     [7, 3, 5, 6],   # corner 111
                     [0, 3, 5, 6]],  # middle tet
                    dtype=np.int64)


def _orient(X, tets):
    """Reorder vertices so every tet has positive signed volume."""
    a, b, c, d = (X[tets[:, i]] for i in range(4))
    det = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    neg = det < 0
    tets = tets.copy()
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return tets


def voxel_mesh(keep, h=1.0, origin=(0.0, 0.0, 0.0)):
    """Tet mesh of the kept cubes of a boolean voxel grid.

    keep: bool array [nx, ny, nz]; cube (i, j, k) spans
    origin + h * ([i, i+1] x [j, j+1] x [k, k+1]).
    Returns (X [n, 3] float64, tets [E, 4] int32, grid_index [n, 3] int64).
    """
    keep = np.asarray(keep, dtype=bool)
    nx, ny, nz = keep.shape
    ci, cj, ck = np.nonzero(keep)
    corner = np.array([[b & 1, (b >> 1) & 1, (b >> 2) & 1] for b in range(8)])
    # node id of each cube corner in the (nx+1)(ny+1)(nz+1) lattice
    lat = ((ci[:, None] + corner[None, :, 0]) * (ny + 1)
           + (cj[:, None] + corner[None, :, 1])) * (nz + 1) + (ck[:, None] + corner[None, :, 2])
    used, inv = np.unique(lat.ravel(), return_inverse=True)
    cube_nodes = inv.reshape(lat.shape)
    par = (ci + cj + ck) & 1
    tets = np.empty((len(ci), 5, 4), dtype=np.int64)
    tets[par == 0] = cube_nodes[par == 0][:, _SPLIT_A]
    tets[par == 1] = cube_nodes[par == 1][:, _SPLIT_B]
    tets = tets.reshape(-1, 4)
    gk = used % (nz + 1)
    gj = (used // (nz + 1)) % (ny + 1)
    gi = used // ((nz + 1) * (ny + 1))
    gidx = np.stack([gi, gj, gk], axis=1)
    X = np.asarray(origin, dtype=np.float64)[None, :] + h * gidx.astype(np.float64)
    tets = _orient(X, tets)
    return X, tets.astype(np.int32), gidx


def grid_mesh(nx, ny, nz, h=1.0, origin=(0.0, 0.0, 0.0)):
    """Box of nx * ny * nz cubes, five tets per cube."""
    return voxel_mesh(np.ones((nx, ny, nz), dtype=bool), h, origin)


def boundary_faces(tets):
    """Triangles that belong to exactly one tet, as [F, 3] node ids."""
    faces = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]],
                            tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]])
    key = np.sort(faces, axis=1)
    _, idx, cnt = np.unique(key, axis=0, return_index=True, return_counts=True)
    return faces[idx[cnt == 1]]


def boundary_faces_outward(X, tets):
    """Boundary triangles [F, 3] wound so that (b - a) x (c - a) points out of
    the mesh: for a positively oriented tet (0, 1, 2, 3) the faces (0, 2, 1),
    (0, 1, 3), (0, 3, 2) and (1, 2, 3) face away from the opposite vertex."""
    tets = _orient(X, np.asarray(tets, dtype=np.int64))
    faces = np.concatenate([tets[:, [0, 2, 1]], tets[:, [0, 1, 3]],
                            tets[:, [0, 3, 2]], tets[:, [1, 2, 3]]])
    key = np.sort(faces, axis=1)
    _, idx, cnt = np.unique(key, axis=0, return_index=True, return_counts=True)
    return faces[np.sort(idx[cnt == 1])].astype(np.int32)


def boundary_nodes(tets, n):
    """Boolean mask of nodes on the mesh boundary."""
    mask = np.zeros(n, dtype=bool)
    mask[boundary_faces(tets).ravel()] = True
    return mask


def node_adjacency(tets, n):
    """CSR (indptr, indices) of the node graph (edges of the tets)."""
    pairs = np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(4) if a != b])
    key = np.unique(pairs[:, 0].astype(np.int64) * n + pairs[:, 1])
    rows, cols = key // n, key % n
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    return np.cumsum(indptr), cols


def jitter_interior(X, tets, amount, seed, h=1.0):
    """Move interior nodes by U(-amount, amount)^3 * h; boundary stays planar."""
    rng = np.random.Generator(np.random.PCG64(seed))
    interior = ~boundary_nodes(tets, len(X))
    X = X.copy()
    X[interior] += h * rng.uniform(-amount, amount, size=(int(interior.sum()), 3))
    return X
