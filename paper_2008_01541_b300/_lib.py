"""ctypes declarations of the C ABI in include/pd.h (argument marshalling only)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpd.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libpd.so is not built: run `python -m paper_2008_01541_b300.build` "
                      "(or __graft_entry__.build())")
lib = ctypes.CDLL(LIB_PATH)

FP64, FP32_IR, TF32_IR, BF16_IR, PCG_WARM = 0, 1, 2, 3, 4
STATUS = {0: "PD_OK", 1: "PD_ERR_INVALID_ARG", 2: "PD_ERR_BAD_MESH", 3: "PD_ERR_REGION",
          4: "PD_ERR_CONTACT_OUTSIDE_REGION", 5: "PD_ERR_NOT_SPD", 6: "PD_ERR_NO_CONVERGENCE",
          7: "PD_ERR_TIMEOUT", 8: "PD_ERR_CUDA", 9: "PD_ERR_OOM"}


class PDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("rest_pos", ctypes.c_void_p),
                ("n_tets", ctypes.c_int64), ("tets", ctypes.c_void_p)]


class Material(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("lam", ctypes.c_double), ("density", ctypes.c_double),
                ("mu_prime", ctypes.c_double), ("sigma_min", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("kappa", ctypes.c_double), ("det_min", ctypes.c_double), ("det_max", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("timing", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("n_nodes", "n_tets", "n_free", "n1", "m", "n_alpha", "n_beta", "n_supernodes",
                 "n_levels", "nnz_L", "contacts", "outer_done", "inner_done")] + \
               [("refine_iters", ctypes.c_int), ("residual", ctypes.c_double), ("setup_ms", ctypes.c_double)] + \
               [(name, ctypes.c_double) for name in
                ("ms_local_alpha", "ms_forward", "ms_contact_update", "ms_local_beta", "ms_factor_solve",
                 "ms_bookkeeping", "ms_backward", "ms_step")] + [("kernel_launches", ctypes.c_int64),
                                                                  ("ms_refactor", ctypes.c_double),
                                                                  ("starts_rejected", ctypes.c_int64),
                                                                  ("precision_fallbacks", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)
P = ctypes.c_void_p
I64 = ctypes.c_int64
D = ctypes.c_double

_sigs = {
    "pd_setup": (ctypes.c_int, [ctypes.POINTER(Mesh), ctypes.POINTER(Material), D, P, I64, P, I64,
                                ctypes.POINTER(Options), ctypes.POINTER(P)]),
    "pd_set_dirichlet": (ctypes.c_int, [P, P]),
    "pd_set_contacts": (ctypes.c_int, [P, I64, P, P, P, P]),
    "pd_set_contact_pairs": (ctypes.c_int, [P, I64, P, P, P, P]),
    "pd_set_contact_nodes": (ctypes.c_int, [P, P, I64]),
    "pd_set_detector_spheres": (ctypes.c_int, [P, P, I64, ctypes.c_int, P, D]),
    "pd_set_detector_pairs": (ctypes.c_int, [P, P, I64, P, I64, D, D]),
    "pd_set_detector_triangles": (ctypes.c_int, [P, P, I64, P, I64, P, I64, P, I64, D, D, D]),
    "pd_clear_detector": (ctypes.c_int, [P]),
    "pd_detect": (ctypes.c_int, [P]),
    "pd_get_contacts": (ctypes.c_int, [P, I64, ctypes.POINTER(I64), P, P, P, P]),
    "pd_step": (ctypes.c_int, [P, ctypes.c_int, CB, P]),
    "pd_get_positions": (ctypes.c_int, [P, P]),
    "pd_get_positions_dev": (ctypes.c_int, [P, P]),
    "pd_get_state": (ctypes.c_int, [P, P, P]),
    "pd_set_state": (ctypes.c_int, [P, P, P]),
    "pd_get_stats": (ctypes.c_int, [P, ctypes.POINTER(Stats)]),
    "pd_last_error": (ctypes.c_char_p, [P]),
    "pd_destroy": (None, [P]),
    "pd_local_step": (ctypes.c_int, [P, P, P, P]),
    "pd_get_schur": (ctypes.c_int, [P, P]),
    "pd_schur_solve": (ctypes.c_int, [P, P, P, P]),
    "pd_schur_solve_dev": (ctypes.c_int, [P, P, P, P]),
    "pd_set_precision": (ctypes.c_int, [P, ctypes.c_int]),
    "pd_set_inner_iters": (ctypes.c_int, [P, ctypes.c_int]),
    "pd_debug_wait_timeout": (ctypes.c_int, [P]),
    "pd_set_warm_start": (ctypes.c_int, [P, ctypes.c_int]),
    "pd_set_pcg_capacitance": (ctypes.c_int, [P, ctypes.c_int]),
    "pd_set_precision_fallback": (ctypes.c_int, [P, ctypes.c_int]),
    "pd_mlp_set_params": (ctypes.c_int, [P, P, I64]),
    "pd_mlp_get_params": (ctypes.c_int, [P, P, I64]),
    "pd_mlp_record": (ctypes.c_int, [P, I64]),
    "pd_mlp_train": (ctypes.c_int, [P, I64, I64, D, ctypes.c_uint64, ctypes.POINTER(D)]),
    "pd_mlp_eval": (ctypes.c_int, [P, ctypes.POINTER(D), ctypes.POINTER(D)]),
    "pd_mlp_set_loss": (ctypes.c_int, [P, ctypes.c_int]),
    "pd_mlp_loss_grad": (ctypes.c_int, [P, P, P, I64, ctypes.POINTER(D), P]),
    "pd_tc_rank_k": (ctypes.c_int, [ctypes.c_int, P, P, P, I64, I64, I64, P]),
    "pd_schur_solve_noalloc": (ctypes.c_int, [P, I64, I64, P, P, P, P, P, P, ctypes.c_char_p, I64]),
    "pd_host_schur": (ctypes.c_int, [ctypes.POINTER(Mesh), ctypes.POINTER(Material), D, P, I64, P, I64,
                                     P, ctypes.c_char_p, I64]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(_sigs)
MLP_NPARAMS = 136195
