"""ctypes view of libsp2.so (the C ABI declared in include/sp2.h).

Loading fails loudly: if the shared library has not been built there is no
fallback of any kind. Build it with ``paper_2409_17033_gb300.build.build()``
(or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsp2.so")

SP2_MAX_ITER = 256

# sp2_status
OK, EINVAL, ENOMEM, ENOCONV, ENONFINITE, ETIMEOUT, ECUDA, ENOTIMPL, ENOSTATE = range(9)
STATUS_NAMES = {0: "SP2_OK", 1: "SP2_EINVAL", 2: "SP2_ENOMEM", 3: "SP2_ENOCONV",
                4: "SP2_ENONFINITE", 5: "SP2_ETIMEOUT", 6: "SP2_ECUDA", 7: "SP2_ENOTIMPL",
                8: "SP2_ENOSTATE"}

# sp2_dtype
F64, F32 = 0, 1
# sp2_mode
MODE_FP64, MODE_FP32, MODE_BF16X2, MODE_FP16X2, MODE_BF16X3, MODE_BF16_TAIL = 0, 1, 2, 3, 4, 5
MODES = {"fp64": MODE_FP64, "fp32": MODE_FP32, "bf16x2": MODE_BF16X2, "fp16x2": MODE_FP16X2,
         "bf16x3": MODE_BF16X3, "bf16_tail": MODE_BF16_TAIL}
DEFAULT_TAIL_F = 1.0   # SP2_DEFAULT_TAIL_F
CKPT_AUTO = -1   # SP2_CKPT_AUTO
# sp2_option
OPTION_WAIT_LIMIT_NS, OPTION_WITHHOLD_LOAD, OPTION_FUSED_RESPONSE, OPTION_PAIR_TILES = 0, 1, 2, 3


class Opts(C.Structure):
    _fields_ = [
        ("mode", C.c_int),
        ("idem_tol", C.c_double),
        ("floor_gate", C.c_double),
        ("max_iter", C.c_int),
        ("min_iter", C.c_int),
        ("fixed_m", C.c_int),
        ("sigma_in", C.POINTER(C.c_int8)),
        ("eps_min", C.c_double),
        ("eps_max", C.c_double),
        ("ckpt_k", C.c_int),
        ("keep_history", C.c_int),
        ("time_kernels", C.c_int),
        ("tail_f", C.c_double),
        ("block_sparse", C.c_int),
        ("block_tau", C.c_double),
    ]


class Info(C.Structure):
    _fields_ = [
        ("M", C.c_int),
        ("converged", C.c_int),
        ("alpha", C.c_double),
        ("beta", C.c_double),
        ("eps_min", C.c_double),
        ("eps_max", C.c_double),
        ("trace", C.c_double),
        ("idem_err", C.c_double),
        ("sigma", C.c_int8 * SP2_MAX_ITER),
        ("errors", C.c_double * (SP2_MAX_ITER + 1)),
        ("idem_fro", C.c_double * SP2_MAX_ITER),
        ("n_gemm_launches", C.c_int64),
        ("executed_flops", C.c_double),
        ("algorithmic_flops", C.c_double),
        ("kernel_launches", C.c_int64),
        ("product_ms", C.c_double),
        ("product_launches_timed", C.c_int64),
        ("ckpt_k", C.c_int),
        ("refine_iter", C.c_int),
        ("tail_single_steps", C.c_int),
        ("block_fill", C.c_double),
    ]

    def to_dict(self) -> dict:
        m = self.M
        return {
            "M": m,
            "converged": bool(self.converged),
            "alpha": self.alpha,
            "beta": self.beta,
            "eps_min": self.eps_min,
            "eps_max": self.eps_max,
            "trace": self.trace,
            "idem_err": self.idem_err,
            "sigma": [int(self.sigma[i]) for i in range(m)],
            "errors": [float(self.errors[i]) for i in range(m + 1)],
            "idem_fro": [float(self.idem_fro[i]) for i in range(m)],
            "n_gemm_launches": int(self.n_gemm_launches),
            "executed_flops": float(self.executed_flops),
            "algorithmic_flops": float(self.algorithmic_flops),
            "kernel_launches": int(self.kernel_launches),
            "product_ms": float(self.product_ms),
            "product_launches_timed": int(self.product_launches_timed),
            "ckpt_k": int(self.ckpt_k),
            "refine_iter": int(self.refine_iter),
            "tail_single_steps": int(self.tail_single_steps),
            "block_fill": float(self.block_fill),
        }


class ScfOpts(C.Structure):
    _fields_ = [
        ("mixer", C.c_int),
        ("alpha", C.c_double),
        ("history", C.c_int),
        ("tol", C.c_double),
        ("max_iter", C.c_int),
        ("W1", C.c_void_p),
        ("W2", C.c_void_p),
        ("hidden", C.c_int),
        ("bf16_infer", C.c_int),
        ("refine_mode", C.c_int),
        ("refine_below", C.c_double),
        ("kT", C.c_double),
        ("mu", C.c_double),
        ("n_doublings", C.c_int),
        ("canonical", C.c_int),
    ]


MIXERS = {"linear": 0, "anderson": 1, "mlp": 2, "anderson_mlp": 3}

EXPORTS = {
    "sp2_default_opts": (None, [C.POINTER(Opts)]),
    "sp2_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.c_size_t]),
    "sp2_destroy": (C.c_int, [C.c_void_p]),
    "sp2_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sp2_last_error": (C.c_char_p, [C.c_void_p]),
    "sp2_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int64]),
    "sp2_workspace_bytes": (C.c_size_t, [C.c_void_p]),
    "sp2_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double,
                              C.POINTER(Opts), C.c_void_p, C.POINTER(Info)]),
    "sp2_response": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double,
                               C.c_void_p, C.c_int64, C.c_int, C.POINTER(Opts), C.c_void_p,
                               C.c_void_p, C.POINTER(Info)]),
    "sp2_susceptibility": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double,
                                     C.c_void_p, C.c_int64, C.c_int, C.c_int, C.POINTER(Opts),
                                     C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    "sp2_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                              C.POINTER(Info)]),
    "sp2_release_history": (C.c_int, [C.c_void_p]),
    "sp2_synchronize": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "sp2_fermi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_double,
                            C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.POINTER(Opts),
                            C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    "sp2_nonorth_susceptibility": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                             C.c_double, C.c_void_p, C.POINTER(Opts), C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    "response_contract": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_int64, C.c_int, C.c_int, C.c_void_p]),
    "sp2_scf_response": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_int,
                                   C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(ScfOpts),
                                   C.POINTER(Opts), C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.POINTER(Info)]),
    "sp2_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                  C.c_int64, C.c_void_p, C.c_int]),
    "sp2_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                                    C.c_void_p, C.c_void_p]),
    "sp2_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_void_p]),
    "response_contract_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                            C.c_int64, C.c_int, C.c_int, C.c_void_p,
                                            C.c_void_p]),
}

_lib = None


def load() -> C.CDLL:
    """Load libsp2.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libsp2.so not found at {LIB_PATH}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()'). There is no CPU fallback.")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SP2Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
