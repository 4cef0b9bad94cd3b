"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    try:
        import torch
        if not torch.cuda.is_available():
            pytest.skip("no CUDA device")
    except ImportError:
        pytest.skip("torch missing")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def contact_tuple(c):
    return (c.nodes, c.w, c.target, c.stiffness)


def region_callback(scene, step, ref_x):
    """Adapter: the library hands x_2 (region order); the scene wants full x."""
    def fn(x2):
        x = ref_x.copy()
        x[scene.region] = x2
        return contact_tuple(scene.contacts(step, x))
    return fn


def oracle_callback(scene, step):
    def fn(x):
        return scene.contacts(step, x)
    return fn


def parity_errors(xg, xo, x0):
    """(norm error, per-node error) of a GPU result xg against the oracle's
    xo, both relative to the oracle's displacement from x0: the norm error is
    ||xg - xo|| / ||xo - x0||, the per-node error max_i |xg_i - xo_i| /
    max_i |xo_i - x0_i| over the nodes' position vectors."""
    d = np.linalg.norm(xo - x0)
    dn = np.linalg.norm(xo - x0, axis=1).max()
    return (np.linalg.norm(xg - xo) / d if d > 0 else np.linalg.norm(xg - xo),
            np.linalg.norm(xg - xo, axis=1).max() / dn if dn > 0 else np.linalg.norm(xg - xo, axis=1).max())


def assert_parity(xg, xo, x0, tol, what=""):
    """Both the norm and the per-node error of xg against xo within tol."""
    e, en = parity_errors(xg, xo, x0)
    assert e <= tol and en <= tol, (what, e, en)
    return e, en
