"""Driving the learned warm start: generate training solves with the method
itself along seeded random indenter paths, train the network on the device,
and compare PCG iteration counts by starting point.  Host orchestration only;
every solve, feature and gradient is computed by libpd.so."""
import time

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


def _paths(scene, n_solves, seed, path_len, radius):
    """Seeded indenter paths of path_len steps covering n_solves steps."""
    out = []
    k = 0
    while sum(len(p) for p in out) < n_solves:
        c, _ = indenter_path(scene, seed=seed * 100003 + k, steps=min(path_len, n_solves - sum(len(p) for p in out)),
                             radius=radius)
        out.append(c)
        k += 1
    return out


def _run_paths(solver, scene, state, paths, radius, depth):
    iters = []
    for p in paths:
        solver.set_state(*state)
        iters += run_path(solver, scene, p, radius, depth=depth)
    return iters


def config5(solver, scene, state, n_train=18000, n_val=1000, n_test=1000, path_len=200, radius_h=10.0,
            depth=0.25, loss=1, epochs=4.0, batch=4096, lr=1e-3, seed=0, timer=None):
    """The learned warm start as configuration 5 specifies it: region solves
    generated by the method itself (split-TF32 refactorisation, 1 outer x 1
    inner iteration per step) along seeded random indenter paths, split into
    training / validation / test solves on disjoint paths; the network
    trained on the device; then every test path run with PCG from each
    starting point (zero, previous solution, z0, network), with the
    contact-free preconditioner M0 alone and with its capacitance correction,
    and with plain refactorisation, reporting iterations and time per step.  `state` is the
    (x, v) every path starts from; `timer(fn)` returns the device ms of fn().
    Host orchestration only: every solve, feature and gradient runs in the
    library."""
    from . import _lib as L
    h = scene.info.get("h", 1.0)
    radius = radius_h * h
    tr = _paths(scene, n_train, seed + 1, path_len, radius)
    va = _paths(scene, n_val, seed + 2, path_len, radius)
    te = _paths(scene, n_test, seed + 3, path_len, radius)
    out = {"solves": {"train": n_train, "val": n_val, "test": n_test}, "indenter_radius": radius,
           "depth": depth, "loss": ["mse", "diag_energy"][loss]}
    solver.set_precision(L.FP32_IR)
    solver.mlp_set_loss(loss)
    solver.mlp_set_params(he_init(seed))
    solver.mlp_record(n_train)
    t0 = time.perf_counter()
    _run_paths(solver, scene, state, tr, radius, depth)
    out["generate_s"] = time.perf_counter() - t0
    rows = n_train * solver.m
    steps = int(max(1, epochs * rows / batch))
    t0 = time.perf_counter()
    out["train_loss"] = solver.mlp_train(steps, batch=batch, lr=lr, seed=seed + 7)
    out["train_s"] = time.perf_counter() - t0
    out["train_steps"], out["epochs"] = steps, epochs
    solver.mlp_record(n_val)
    _run_paths(solver, scene, state, va, radius, depth)
    net, zero = solver.mlp_eval()
    out["val_err_network_vs_z0"] = net / zero if zero > 0 else None
    solver.mlp_record(0)
    by = {}
    runs = [("refactor (split-TF32 + IR)", L.FP32_IR, 0, True)]
    for cap, tag in ((False, "pcg M0"), (True, "pcg M0 + capacitance")):
        runs += [(tag + " zero", L.PCG_WARM, 0, cap), (tag + " previous", L.PCG_WARM, 1, cap),
                 (tag + " z0", L.PCG_WARM, 3, cap), (tag + " network", L.PCG_WARM, 2, cap)]
    for name, prec, src, cap in runs:
        solver.set_precision(prec)
        solver.set_pcg_capacitance(cap)
        solver.set_warm_start(src)
        its = []
        rej0 = solver.stats()["starts_rejected"]
        ms = timer(lambda: its.extend(_run_paths(solver, scene, state, te, radius, depth))) if timer else None
        by[name] = {"iterations": float(np.mean(its)), "ms_per_step": ms / n_test if ms is not None else None,
                    "starts_rejected": int(solver.stats()["starts_rejected"] - rej0)}
    solver.set_warm_start(0)
    solver.set_pcg_capacitance(True)
    solver.set_precision(L.FP64)
    out["test"] = by
    return out
