"""Seeded synthetic scenes shaped like the paper's workloads (Section 4).

This module only builds inputs: rest meshes, Dirichlet sets, the collision-prone
node set and the obstacle queries that turn current proxy positions into
penalty springs.  It holds none of the solver's arithmetic, and both the FP64
oracle and the CUDA library are fed from it.
"""
from .mesh import grid_mesh, voxel_mesh, boundary_nodes, boundary_faces_outward, node_adjacency
from .configs import (Scene, Contacts, config1, elbow, slabs, small_elbow,
                      tiny_cube, sphere_contacts, cylinder_contacts,
                      empty_contacts, rotation_z, pair_contacts, closed_pose)

__all__ = ["grid_mesh", "voxel_mesh", "boundary_nodes", "boundary_faces_outward", "node_adjacency",
           "Scene", "Contacts", "config1", "elbow", "slabs", "small_elbow",
           "tiny_cube", "sphere_contacts", "cylinder_contacts",
           "empty_contacts", "rotation_z", "pair_contacts", "closed_pose"]
