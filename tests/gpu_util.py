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
