"""ctypes declarations of ``liblbm.so`` (the C ABI in ``include/lbm.h``).

Argument marshalling only.  The library is loaded from this package's
directory; if it has not been built the import fails loudly - there is no
fallback implementation.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the same ABI (e.g. the checked build,
# compiled with -DLBM_CHECKED); default: the package's liblbm.so.
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE, LBM_ECHECK = (
    0, -1, -2, -3, -4, -5, -6, -7)
LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S = 0, 1, 2, 3
LBM_WALL_BOUNCEBACK, LBM_WALL_ELASTIC_GZS = 0, 1
LBM_IOLET_VELOCITY, LBM_IOLET_DENSITY = 0, 1
LBM_PROFILE_PARABOLIC, LBM_PROFILE_WOMERSLEY, LBM_PROFILE_PLUG = 0, 1, 2

# Every symbol include/lbm.h and include/lbm_mlp.h declare.
EXPORTS = (
    "lbm_build_lattice", "lbm_set_wall_params", "lbm_init_fields", "lbm_step", "lbm_step_diag",
    "lbm_moments",
    "lbm_sync", "lbm_info", "lbm_export_lattice", "lbm_wall_state", "lbm_reduce",
    "lbm_get_populations", "lbm_set_populations", "lbm_checkpoint_bytes", "lbm_checkpoint_save",
    "lbm_checkpoint_load", "lbm_wss", "lbm_set_stream", "lbm_last_error", "lbm_status_string",
    "lbm_destroy", "lbm_profile", "lbm_profile_read", "lbm_reduce_noalloc",
    "lbm_ensemble_create", "lbm_ensemble_step", "lbm_ensemble_sync", "lbm_ensemble_tune",
    "lbm_ensemble_last_error", "lbm_ensemble_destroy", "lbm_fmap", "lbm_plan_lattice", "lbm_tune",
    # include/lbm_mlp.h
    "lbm_mlp_create", "lbm_mlp_param_count", "lbm_mlp_set_params", "lbm_mlp_get_params",
    "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_train_step", "lbm_mlp_sync",
    "lbm_mlp_last_error", "lbm_mlp_destroy", "lbm_warm_features", "lbm_warm_start",
)
LBM_TUNE_PREFETCH, LBM_TUNE_SCHEDULE, LBM_TUNE_GRAPH_STEPS = 0, 1, 2
LBM_TUNE_PERSISTENT, LBM_TUNE_BARRIER_EXTRA, LBM_TUNE_BULK_SITES, LBM_TUNE_BULK_WARPS = 3, 4, 5, 6


class LbmIolet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("profile", C.c_int32), ("rho", C.c_double),
                ("u_mean", C.c_double), ("u_amp", C.c_double), ("period", C.c_double),
                ("phase", C.c_double), ("centre", C.c_double * 3), ("axis", C.c_double * 3),
                ("radius", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class LbmAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


LBM_WARM_MAX_GLOBAL = 14


class LbmAdam(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double)]


class LbmWarmFrame(C.Structure):
    _fields_ = [("centre", C.c_double * 3), ("axis", C.c_double * 3), ("z0", C.c_double),
                ("length", C.c_double), ("radius", C.c_double), ("rho_scale", C.c_double),
                ("u_scale", C.c_double), ("n_global", C.c_int32),
                ("global_", C.c_float * LBM_WARM_MAX_GLOBAL)]


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status_name(status), message))
        self.status = status


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbm.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2108_08783_gb300.build" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    i32, i64, dbl = C.c_int32, C.c_int64, C.c_double
    sig = {
        "lbm_build_lattice": ([P, i32, i32, i32, P, i32, i32, dbl, P, P, C.POINTER(P)], C.c_int),
        "lbm_set_wall_params": ([P, i32, dbl, P, P, i64], C.c_int),
        "lbm_init_fields": ([P, P, P], C.c_int),
        "lbm_step": ([P, i64], C.c_int),
        "lbm_step_diag": ([P, i64, P], C.c_int),
        "lbm_moments": ([P, P, P, i32], C.c_int),
        "lbm_sync": ([P], C.c_int),
        "lbm_info": ([P, P], C.c_int),
        "lbm_export_lattice": ([P, P, P, P, P], C.c_int),
        "lbm_wall_state": ([P, P, P], C.c_int),
        "lbm_reduce": ([P, P], C.c_int),
        "lbm_get_populations": ([P, P, i32], C.c_int),
        "lbm_set_populations": ([P, P, i64, i32], C.c_int),
        "lbm_checkpoint_bytes": ([P], C.c_size_t),
        "lbm_checkpoint_save": ([P, P, C.c_size_t], C.c_int),
        "lbm_checkpoint_load": ([P, P, C.c_size_t], C.c_int),
        "lbm_wss": ([P, P, P, i64, P], C.c_int),
        "lbm_set_stream": ([P, P], C.c_int),
        "lbm_tune": ([P, i32, i64], C.c_int),
        "lbm_last_error": ([P], C.c_char_p),
        "lbm_status_string": ([C.c_int], C.c_char_p),
        "lbm_destroy": ([P], None),
        "lbm_profile": ([P, i32], C.c_int),
        "lbm_profile_read": ([P, P, P], C.c_int),
        "lbm_reduce_noalloc": ([P, P, i32], C.c_int),
        "lbm_ensemble_create": ([P, i32, C.POINTER(P)], C.c_int),
        "lbm_ensemble_step": ([P, i64], C.c_int),
        "lbm_ensemble_sync": ([P], C.c_int),
        "lbm_ensemble_tune": ([P, i32, i64], C.c_int),
        "lbm_ensemble_last_error": ([P], C.c_char_p),
        "lbm_ensemble_destroy": ([P], None),
        "lbm_fmap": ([P, i64, P, i64, dbl, dbl, P], C.c_int),
        "lbm_plan_lattice": ([P, i32, i32, i32, P, i32, dbl, P], C.c_int),
        "lbm_mlp_create": ([i32, i32, i32, i32, i64, P, P, C.POINTER(P)], C.c_int),
        "lbm_mlp_param_count": ([P, P], C.c_int),
        "lbm_mlp_set_params": ([P, P, i32], C.c_int),
        "lbm_mlp_get_params": ([P, P, i32], C.c_int),
        "lbm_mlp_forward": ([P, P, i64, P], C.c_int),
        "lbm_mlp_loss_grad": ([P, P, P, i64, P, P, i32], C.c_int),
        "lbm_mlp_train_step": ([P, P, P, i64, P, P], C.c_int),
        "lbm_mlp_sync": ([P], C.c_int),
        "lbm_mlp_last_error": ([P], C.c_char_p),
        "lbm_mlp_destroy": ([P], None),
        "lbm_warm_features": ([P, P, P, P], C.c_int),
        "lbm_warm_start": ([P, P, P], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def status_name(status):
    return lib().lbm_status_string(int(status)).decode()


def check(rc, ctx=None):
    if rc != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode()
        raise LbmError(rc, msg)
    return rc
