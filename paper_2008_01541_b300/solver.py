"""Thin Python wrapper over the C ABI: numpy (host) or torch (device) buffers in,
status codes turned into exceptions.  No arithmetic of the method happens here."""
import ctypes
import numpy as np

from . import _lib
from ._lib import lib, PDError


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _mesh(X, tets):
    X = _c(X, np.float64)
    tets = _c(tets, np.int32)
    return _lib.Mesh(len(X), X.ctypes.data, len(tets), tets.ctypes.data), (X, tets)


def host_schur(X, tets, region, dirichlet, mu, density=0.0, dt=0.0, mu_prime=0.0, kappa=0.0):
    """Sigma_0 from the library's host partial Cholesky (no GPU needed)."""
    mesh, keep = _mesh(X, tets)
    region = _c(region, np.int32)
    dirichlet = _c(dirichlet, np.int32)
    mat = _lib.Material(mu, 0.0, density, mu_prime, 0.0, np.inf, kappa, 1.0, 1.0)
    out = np.zeros((len(region), len(region)))
    info = ctypes.create_string_buffer(1024)
    st = lib.pd_host_schur(ctypes.byref(mesh), ctypes.byref(mat), dt, _ptr(region), len(region),
                           _ptr(dirichlet), len(dirichlet), _ptr(out), info, 1024)
    if st:
        raise PDError(st, info.value.decode())
    return out, info.value.decode()


class Solver:
    """One scene on the current CUDA device (pd_setup ... pd_destroy)."""

    def __init__(self, X, tets, region, dirichlet, mu, lam=0.0, density=0.0, dt=0.0,
                 precision=_lib.FP64, inner_iters=1, tol=1e-10, max_refine=50, stream=None, timing=False,
                 mu_prime=0.0, sigma_min=0.0, sigma_max=np.inf, kappa=0.0, det_min=1.0, det_max=1.0):
        mesh, keep = _mesh(X, tets)
        self.n = len(keep[0])
        self.E = len(keep[1])
        self.region = _c(region, np.int32)
        self.dirichlet = _c(dirichlet, np.int32)
        self.m = len(self.region)
        self.nd = len(self.dirichlet)
        mat = _lib.Material(mu, lam, density, mu_prime, sigma_min, sigma_max, kappa, det_min, det_max)
        opt = _lib.Options(precision, tol, max_refine, inner_iters,
                           ctypes.c_void_p(stream) if stream else None, 1 if timing else 0)
        h = ctypes.c_void_p()
        st = lib.pd_setup(ctypes.byref(mesh), ctypes.byref(mat), dt, _ptr(self.region), self.m,
                          _ptr(self.dirichlet), self.nd, ctypes.byref(opt), ctypes.byref(h))
        if st:
            raise PDError(st, lib.pd_last_error(None).decode())
        self.h = h
        self._cb_keep = None

    def _check(self, st):
        if st:
            raise PDError(st, lib.pd_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib.pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_dirichlet(self, pos):
        pos = _c(pos, np.float64).reshape(self.nd, 3)
        self._check(lib.pd_set_dirichlet(self.h, _ptr(pos)))

    def set_contacts(self, nodes, w, target, stiffness):
        """Springs with 4 node slots (one proxy) or 8 (two-sided, pd_set_contact_pairs)."""
        nodes = np.asarray(nodes)
        slots = 8 if nodes.ndim == 2 and nodes.shape[1] == 8 else 4
        nodes = _c(nodes, np.int32).reshape(-1, slots)
        k = len(nodes)
        w = _c(w, np.float64).reshape(k, slots)
        target = _c(target, np.float64).reshape(k, 3)
        stiffness = _c(stiffness, np.float64).reshape(k)
        fn = lib.pd_set_contact_pairs if slots == 8 else lib.pd_set_contacts
        self._check(fn(self.h, k, _ptr(nodes), _ptr(w), _ptr(target), _ptr(stiffness)))

    def set_contact_nodes(self, nodes):
        """Nested Schur refactorisation of the FP64 form on these contact nodes
        (None or empty: off)."""
        a = _c(nodes if nodes is not None else np.zeros(0), np.int32)
        self._check(lib.pd_set_contact_nodes(self.h, _ptr(a) if len(a) else None, len(a)))

    def set_detector_spheres(self, proxies, spheres, stiffness):
        proxies = _c(proxies, np.int32)
        spheres = _c(spheres, np.float64).reshape(-1, 4)
        self._check(lib.pd_set_detector_spheres(self.h, _ptr(proxies), len(proxies), len(spheres), _ptr(spheres),
                                                float(stiffness)))

    def set_detector_pairs(self, side_a, side_b, gap, stiffness):
        a = _c(side_a, np.int32)
        b = _c(side_b, np.int32)
        self._check(lib.pd_set_detector_pairs(self.h, _ptr(a), len(a), _ptr(b), len(b), float(gap), float(stiffness)))

    def set_detector_triangles(self, prox_a, tris_a, prox_b, tris_b, gap, rest_min, stiffness):
        """Point-triangle self-contact: side-A nodes against side-B triangles
        and side-B nodes against side-A triangles (outward-wound [nt, 3])."""
        pa, pb = _c(prox_a, np.int32), _c(prox_b, np.int32)
        ta, tb = _c(tris_a, np.int32).reshape(-1, 3), _c(tris_b, np.int32).reshape(-1, 3)
        self._check(lib.pd_set_detector_triangles(self.h, _ptr(pa), len(pa), _ptr(ta), len(ta), _ptr(pb), len(pb),
                                                  _ptr(tb), len(tb), float(gap), float(rest_min), float(stiffness)))

    def detect(self):
        """Run the device detector once on the current positions."""
        self._check(lib.pd_detect(self.h))

    def contacts(self):
        """The active spring slots: (nodes [k,8], w [k,8], target [k,3], stiffness [k])."""
        k = ctypes.c_int64()
        self._check(lib.pd_get_contacts(self.h, 0, ctypes.byref(k), None, None, None, None))
        n = k.value
        nodes = np.empty((n, 8), np.int32)
        w = np.empty((n, 8))
        t = np.empty((n, 3))
        c = np.empty(n)
        if n:
            self._check(lib.pd_get_contacts(self.h, n, ctypes.byref(k), _ptr(nodes), _ptr(w), _ptr(t), _ptr(c)))
        return nodes, w, t, c

    def clear_detector(self):
        self._check(lib.pd_clear_detector(self.h))

    def step(self, outer_iters, contacts_fn=None):
        """contacts_fn(x2 [m,3] numpy) -> (nodes, w, target, stiffness) or None."""
        if contacts_fn is None:
            self._check(lib.pd_step(self.h, outer_iters, _lib.CB(), None))
            return
        m = self.m
        err = []

        def cb(user, x2p, handle):
            try:
                x2 = np.ctypeslib.as_array(x2p, shape=(m, 3)).copy()
                c = contacts_fn(x2)
                if c is not None:
                    self.set_contacts(*c)
                return 0
            except PDError as e:
                err.append(e)
                return e.code
            except Exception as e:  # pragma: no cover - surfaced below
                err.append(e)
                return 1

        fn = _lib.CB(cb)
        st = lib.pd_step(self.h, outer_iters, fn, None)
        if err:
            raise err[0]
        self._check(st)

    def positions(self):
        out = np.empty((self.n, 3))
        self._check(lib.pd_get_positions(self.h, _ptr(out)))
        return out

    def positions_dev(self, out):
        self._check(lib.pd_get_positions_dev(self.h, _dptr(out)))
        return out

    def get_state(self):
        x = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        self._check(lib.pd_get_state(self.h, _ptr(x), _ptr(v)))
        return x, v

    def set_state(self, x, v=None):
        x = _c(x, np.float64)
        v = None if v is None else _c(v, np.float64)
        self._check(lib.pd_set_state(self.h, _ptr(x), _ptr(v) if v is not None else None))

    def stats(self):
        st = _lib.Stats()
        self._check(lib.pd_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def local_step(self, x, want_R=True):
        x = _c(x, np.float64)
        R = np.empty((self.E, 3, 3)) if want_R else None
        f = np.empty((self.n, 3))
        self._check(lib.pd_local_step(self.h, _ptr(x), _ptr(R) if want_R else None, _ptr(f)))
        return R, f

    def schur(self):
        out = np.empty((self.m, self.m))
        self._check(lib.pd_get_schur(self.h, _ptr(out)))
        return out

    def schur_solve(self, g, u0=None):
        g = _c(g, np.float64).reshape(self.m, 3)
        u = np.empty((self.m, 3))
        u0 = None if u0 is None else _c(u0, np.float64).reshape(self.m, 3)
        self._check(lib.pd_schur_solve(self.h, _ptr(g), _ptr(u0) if u0 is not None else None, _ptr(u)))
        return u

    def schur_solve_dev(self, g, u, u0=None):
        self._check(lib.pd_schur_solve_dev(self.h, _dptr(g), _dptr(u0), _dptr(u)))
        return u

    def set_precision(self, p):
        self._check(lib.pd_set_precision(self.h, p))

    def set_inner_iters(self, n):
        self._check(lib.pd_set_inner_iters(self.h, int(n)))

    # ---- learned warm start (PD_PCG_WARM) ----
    def set_warm_start(self, source):
        """0 = zero, 1 = previous region solution, 2 = network prediction, 3 = z0."""
        self._check(lib.pd_set_warm_start(self.h, int(source)))

    def set_pcg_capacitance(self, on):
        """Capacitance (Woodbury) correction of the PCG preconditioner for the active springs."""
        self._check(lib.pd_set_pcg_capacitance(self.h, 1 if on else 0))

    def set_precision_fallback(self, on):
        """Redo a failed low-precision region solve by the FP64 factorisation (on by default)."""
        self._check(lib.pd_set_precision_fallback(self.h, 1 if on else 0))

    def mlp_set_params(self, params):
        p = _c(params, np.float32).ravel()
        self._check(lib.pd_mlp_set_params(self.h, _ptr(p), len(p)))

    def mlp_get_params(self):
        p = np.empty(_lib.MLP_NPARAMS, np.float32)
        self._check(lib.pd_mlp_get_params(self.h, _ptr(p), len(p)))
        return p

    def mlp_record(self, max_solves):
        self._check(lib.pd_mlp_record(self.h, int(max_solves)))

    def mlp_train(self, steps, batch=1024, lr=1e-3, seed=0):
        loss = ctypes.c_double()
        self._check(lib.pd_mlp_train(self.h, int(steps), int(batch), float(lr), int(seed), ctypes.byref(loss)))
        return loss.value

    def mlp_loss_grad(self, X, T):
        X = _c(X, np.float32)
        T = _c(T, np.float32)
        grad = np.empty(_lib.MLP_NPARAMS, np.float32)
        loss = ctypes.c_double()
        self._check(lib.pd_mlp_loss_grad(self.h, _ptr(X), _ptr(T), len(X), ctypes.byref(loss), _ptr(grad)))
        return loss.value, grad

    def mlp_set_loss(self, kind):
        """0: mean squared error; 1: rows weighted by H_ii (diagonal energy norm)."""
        self._check(lib.pd_mlp_set_loss(self.h, int(kind)))

    def mlp_eval(self):
        """(mse of the network, mse of the zero prediction) over the recorded rows."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(lib.pd_mlp_eval(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value
