"""ctypes view of include/p4d.h and the loader of libp4d.so.

The library is built in-tree by ``paper_2602_07225_gb300.build``; there is no
fallback implementation: if the shared library cannot be loaded every call
raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libp4d.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory", 4: "not converged",
          5: "Krylov breakdown", 6: "non-finite value", 7: "concentration outside the kinetics domain",
          8: "device wait timed out"}
OK, INVALID_ARG, CUDA_ERR, OOM, NOT_CONVERGED, BREAKDOWN, NONFINITE, DOMAIN, TIMEOUT = range(9)


class P4DError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, STATUS.get(status, "?"), status))


_dp = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("hx", _dp), ("hy", _dp), ("hz", _dp), ("region", _u8p), ("eps", _dp), ("eps_s", _dp),
                ("Rs", _dp), ("Ds", _dp), ("gamma_p", _u8p), ("gamma_n", _u8p), ("rgrid", _dp),
                ("nc", C.c_int32), ("sigma_e", _dp), ("Ds_e", _dp), ("shell_sigma_t_p", C.c_double),
                ("shell_sigma_t_n", C.c_double)]


class Params(C.Structure):
    _fields_ = [("F", C.c_double), ("R", C.c_double), ("T", C.c_double), ("tplus", C.c_double),
                ("brug", C.c_double), ("De", C.c_double), ("kappa", C.c_double),
                ("sigma_n", C.c_double), ("sigma_p", C.c_double), ("k_n", C.c_double), ("k_p", C.c_double),
                ("cmax_n", C.c_double), ("cmax_p", C.c_double), ("alpha", C.c_double),
                ("ocp_n", C.c_double * 2), ("ocp_p", C.c_double * 2),
                ("dt", C.c_double), ("i_app", C.c_double), ("diffpot_sign", C.c_double),
                ("precision", C.c_int32), ("combine", C.c_int32), ("order", C.c_int32 * 3),
                ("restart", C.c_int32), ("maxit", C.c_int32), ("mode", C.c_int32),
                ("cheb_degree", C.c_int32), ("coarse_max", C.c_int32), ("cheb_ratio", C.c_double),
                ("rtol", C.c_double), ("profile", C.c_int32), ("ocp_model", C.c_int32),
                ("transport_model", C.c_int32), ("cgs_refine", C.c_int32), ("mf_zchunk", C.c_int32)]


class State(C.Structure):
    _fields_ = [("phis", C.c_void_p), ("phie", C.c_void_p), ("ce", C.c_void_p), ("cs", C.c_void_p),
                ("ce_prev", C.c_void_p), ("cs_prev", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32), ("reorth", C.c_int32),
                ("rel_res", C.c_double), ("rel_res_block", C.c_double * 4), ("ms_total", C.c_double),
                ("ms_precond", C.c_double), ("ms_jvp", C.c_double), ("ms_ortho", C.c_double),
                ("ms_smooth0", C.c_double), ("n_smooth0", C.c_int32), ("n_jvp", C.c_int32),
                ("rel_res_unscaled", C.c_double), ("rel_res_block_unscaled", C.c_double * 4),
                ("nsolves", C.c_int32), ("iters_total", C.c_int32)]

    def as_dict(self):
        return dict(iters=self.iters, restarts=self.restarts, status=self.status, reorth=self.reorth,
                    rel_res=self.rel_res, rel_res_block=list(self.rel_res_block), ms_total=self.ms_total,
                    ms_precond=self.ms_precond, ms_jvp=self.ms_jvp, ms_ortho=self.ms_ortho,
                    ms_smooth0=self.ms_smooth0, n_smooth0=self.n_smooth0, n_jvp=self.n_jvp,
                    rel_res_unscaled=self.rel_res_unscaled,
                    rel_res_block_unscaled=list(self.rel_res_block_unscaled), nsolves=self.nsolves,
                    iters_total=self.iters_total)


# name -> (restype, argtypes); every symbol declared in include/p4d.h
SIGNATURES = {
    "p4d_params_default": (None, [C.POINTER(Params)]),
    "p4d_setup": (C.c_int, [C.POINTER(Mesh), C.POINTER(Params), C.POINTER(State), C.c_void_p, C.POINTER(C.c_void_p)]),
    "p4d_destroy": (None, [C.c_void_p]),
    "p4d_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32)]),
    "p4d_electrode_nodes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "p4d_set_params": (C.c_int, [C.c_void_p, C.POINTER(Params)]),
    "p4d_residual": (C.c_int, [C.c_void_p, C.POINTER(State), C.c_void_p]),
    "p4d_jacobian_update": (C.c_int, [C.c_void_p, C.POINTER(State)]),
    "p4d_jvp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "p4d_precond_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "p4d_fgmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    "p4d_adjoint_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    "p4d_jvp_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "p4d_newton_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_double, C.c_int32, C.POINTER(C.c_int32), C.POINTER(Info)]),
    "p4d_voltage_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "p4d_terminal_voltage": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "p4d_param_grad": (C.c_int, [C.c_void_p, C.POINTER(State), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "p4d_adjoint_prev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "p4d_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "p4d_batch_fgmres_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(Info)]),
    "p4d_batch_adjoint_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(Info)]),
    "p4d_batch_destroy": (None, [C.c_void_p]),
    "p4d_dd_halo_plan": (C.c_int32, [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
    "p4d_dd_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "p4d_dd_set_coarse": (C.c_int, [C.c_void_p, C.c_int32]),
    "p4d_dd_jacobian_update": (C.c_int, [C.c_void_p, C.POINTER(State)]),
    "p4d_dd_jvp": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "p4d_dd_fgmres_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(Info)]),
    "p4d_dd_destroy": (None, [C.c_void_p]),
    "p4d_launch_count": (C.c_longlong, []),
    "p4d_fp64_fma_rate": (C.c_int, [C.POINTER(C.c_double)]),
    "p4d_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libp4d.so (raises OSError if it is missing or does not load)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libp4d.so not built: run paper_2602_07225_gb300.build.build() (%s)" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, where):
    if status != OK:
        raise P4DError(status, where)
