"""Driving the learned warm start: generate training solves with the method
itself along seeded random indenter paths, train the network on the device,
and compare PCG iteration counts by starting point.  Host orchestration only;
every solve, feature and gradient is computed by libpd.so."""
import numpy as np

from . import _lib
from ._lib import PDError  # noqa: F401


def he_init(seed):
    """He-normal weights, zero biases, in the library's logical layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for n, k in [(256, 14), (256, 256), (256, 256), (3, 256)]:
        parts += [rng.normal(0.0, np.sqrt(2.0 / k), size=n * k), np.zeros(n)]
    return np.concatenate(parts).astype(np.float32)


def indenter_path(scene, seed, steps, radius=None, step_len=None):
    """Seeded random walk of a rigid sphere over the collision-prone surface.
    Returns a list of sphere centres (one per time step).  `scene` is any
    object with rest positions X, proxies and an info dict (spacing h)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = scene.X[scene.proxies]
    h = scene.info.get("h", 1.0)
    radius = radius if radius is not None else 4.0 * h
    step_len = step_len if step_len is not None else 0.5 * h
    c = P[rng.integers(len(P))].copy()
    out = []
    for _ in range(steps):
        c = c + step_len * rng.normal(size=3)
        near = P[np.argmin(np.linalg.norm(P - c, axis=1))]
        c = 0.7 * c + 0.3 * near          # stay close to the surface
        out.append(c.copy())
    return out, radius


def run_path(solver, scene, centres, radius, outer=1, depth=0.3):
    """One pd_step per centre with the sphere pushed `depth*radius` into the
    surface; the library's device detector re-detects the proxies inside it
    at every inner iteration (Algorithm 1, step 4.1).  The detector is
    cleared afterwards.  Returns the refinement / PCG iterations per step."""
    iters = []
    try:
        for c in centres:
            sph = np.array([[c[0], c[1], c[2], radius * (1.0 + depth)]], dtype=np.float64)
            solver.set_detector_spheres(scene.proxies, sph, scene.stiffness)
            solver.step(outer)
            iters.append(solver.stats()["refine_iters"])
    finally:
        solver.clear_detector()
    return iters
