"""ctypes binding of liblbhb.so: the C ABI of include/lbhb.h under the same
names.  Argument marshalling only; every step of the lattice update runs in the
library's CUDA kernels.  Loading fails loudly if the library was not built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbhb.so")

LB_OK, LB_ERR_INVALID, LB_ERR_CUDA, LB_ERR_NOMEM = 0, -1, -2, -3
LB_ERR_NONFINITE, LB_ERR_TIMEOUT, LB_ERR_STATE, LB_ERR_UNSUPPORTED = -4, -5, -6, -7
STATUS_NAMES = {0: "LB_OK", -1: "LB_ERR_INVALID", -2: "LB_ERR_CUDA", -3: "LB_ERR_NOMEM",
                -4: "LB_ERR_NONFINITE", -5: "LB_ERR_TIMEOUT", -6: "LB_ERR_STATE",
                -7: "LB_ERR_UNSUPPORTED"}
LB_BC_PERIODIC, LB_BC_COUETTE = 0, 1
LB_FP32, LB_FP16_SHIFTED, LB_FP64, LB_FP16_SHIFTED_SR = 0, 1, 2, 3
LB_KERNEL_AUTO, LB_KERNEL_GENERIC, LB_KERNEL_TILED = 0, 1, 2
LB_SLAB_EDGE_LO, LB_SLAB_EDGE_HI, LB_SLAB_FLOW_LO, LB_SLAB_FLOW_HI = 0, 1, 2, 3

# Every function the header declares, with its ctypes signature.
_D = C.POINTER(C.c_double)
_H = C.c_void_p


class lb_cell_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("tau", C.c_double), ("rho0", C.c_double),
                ("g_aa1", C.c_double), ("g_aa2", C.c_double), ("g_bb1", C.c_double),
                ("g_bb2", C.c_double), ("g_ab", C.c_double), ("u_wall", C.c_double), ("f0", C.c_double),
                ("rho_bar_a", C.c_double), ("rho_bar_b", C.c_double), ("bc", C.c_int), ("tau_b", C.c_double),
                ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double), ("s_nu", C.c_double)]


class mlp_config(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("lam", C.c_double), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("center", C.c_double * 5),
                ("half_range", C.c_double * 5), ("sigma_scale", C.c_double), ("logit_margin", C.c_double)]


_F = C.POINTER(C.c_float)

SIGNATURES = {
    "lb_create": (C.c_int, [C.POINTER(lb_cell_params), C.c_int, C.c_int, C.c_void_p, C.POINTER(_H)]),
    "lb_init_fields": (C.c_int, [_H, _D, _D, _D, _D]),
    "lb_stage_fields": (C.c_int, [_H, _D, _D, _D, _D]),
    "lb_init_fields_staged": (C.c_int, [_H]),
    "lb_set_populations": (C.c_int, [_H, _D]),
    "lb_get_populations": (C.c_int, [_H, _D]),
    "lb_step": (C.c_int, [_H, C.c_longlong]),
    "lb_set_sampling": (C.c_int, [_H, C.c_longlong, C.c_longlong]),
    "lb_shear_stress": (C.c_int, [_H, _D, _D, _D]),
    "lb_get_profile": (C.c_int, [_H, _D, C.POINTER(C.c_longlong)]),
    "lb_get_fields": (C.c_int, [_H, _D, _D, _D, _D]),
    "lb_reductions": (C.c_int, [_H, _D, _D]),
    "lb_set_kernel": (C.c_int, [_H, C.c_int, C.c_int, C.c_int]),
    "lb_autotune": (C.c_int, [_H, C.c_char_p]),
    "lb_get_kernel": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lb_sync": (C.c_int, [_H]),
    "lb_steps_done": (C.c_longlong, [_H]),
    "lb_stream": (C.c_void_p, [_H]),
    "lb_kernel_launches": (C.c_longlong, [_H]),
    "lb_last_error": (C.c_char_p, [_H]),
    "lb_destroy": (None, [_H]),
    "lb_hb_fit": (C.c_int, [_D, _D, C.c_int, C.c_double, C.c_double, _D]),
    "lb_reductions_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                        C.c_void_p]),
    "lb_create_slab": (C.c_int, [C.POINTER(lb_cell_params), C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                 C.POINTER(_H)]),
    "lb_slab_info": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lb_slab_message_bytes": (C.c_int, [_H, C.c_int, C.POINTER(C.c_size_t)]),
    "lb_slab_get": (C.c_int, [_H, C.c_int, C.c_void_p]),
    "lb_slab_put": (C.c_int, [_H, C.c_int, C.c_void_p]),
    "lb_wall_momentum": (C.c_int, [_H, _D, C.POINTER(C.c_longlong)]),
    "lb_launch_shape": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    # include/lbhb_mlp.h
    "mlp_param_count": (C.c_longlong, []),
    "mlp_create": (C.c_int, [C.POINTER(mlp_config), C.c_void_p, C.POINTER(_H)]),
    "mlp_set_params": (C.c_int, [_H, _F, C.c_longlong]),
    "mlp_get_params": (C.c_int, [_H, _F, C.c_longlong]),
    "mlp_forward": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_void_p]),
    "mlp_gradients": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, _F, C.POINTER(C.c_double)]),
    "mlp_train_step": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mlp_serve": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mlp_kernel_launches": (C.c_longlong, [_H]),
    "lb_save": (C.c_int, [_H, C.c_char_p]),
    "lb_test_inject": (C.c_int, [_H, C.c_int]),
    "lb_load": (C.c_int, [_H, C.c_char_p]),
    "mlp_set_error_budget": (C.c_int, [_H, _F, C.c_int, C.c_double, C.c_double, C.c_double]),
    "mlp_destroy": (None, [_H]),
}

_lib = None


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Loads liblbhb.so (built by paper_1004_5058_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbhb.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_1004_5058_gb300.build" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, handle=None):
    if status != LB_OK:
        msg = load().lb_last_error(handle)
        raise LBError(status, msg.decode() if msg else "")
    return status
