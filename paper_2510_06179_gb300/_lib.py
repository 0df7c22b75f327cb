"""ctypes binding of include/dmpc.h (argument marshalling only).

The functions here have the C-ABI's names and signatures; pointers are passed as integers
(device addresses from torch tensors).  Loading fails loudly if the CUDA library has not
been built: there is no fallback path."""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DMPC_LIB") or os.path.join(_PKG, "_build", "libdmpc.so")

c_int, c_float, c_void_p, c_ll = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_longlong
P = c_void_p


class dmpc_ocp_desc(ctypes.Structure):
    _fields_ = [("model", c_int), ("nx", c_int), ("nu", c_int), ("T", c_int), ("dt", c_float),
                ("integrator", c_int)]


class dmpc_options(ctypes.Structure):
    _fields_ = [("sqp_iters", c_int), ("line_search", c_int), ("n_alpha", c_int), ("alpha", c_float * 8),
                ("ls_eta", c_float), ("feas_tol", c_float), ("pcg_tol", c_float), ("pcg_max_iters", c_int),
                ("ru_delta", c_float), ("warm_start", c_int), ("store_schur", c_int),
                ("team_threads", c_int), ("teams_per_block", c_int), ("pcg_precision", c_int),
                ("exact_hessian", c_int), ("pcg_variant", c_int), ("cluster_ctas", c_int)]


SIGNATURES = {
    "dmpc_default_options": (None, [ctypes.POINTER(dmpc_options)]),
    "dmpc_create_problem_batch": (c_int, [ctypes.POINTER(dmpc_ocp_desc), c_int, ctypes.POINTER(dmpc_options),
                                          P, ctypes.POINTER(P)]),
    "dmpc_layout": (c_int, [P, P, P, P, P, P]),
    "dmpc_solve": (c_int, [P, P, P, P, P, P, P, P, P, P, P]),
    "dmpc_vjp": (c_int, [P, P, P, P, P, P, P]),
    "dmpc_solve_plain": (c_int, [P, P, P, P, P, P, P, P, P, P, P]),
    "dmpc_vjp_plain": (c_int, [P, P, P, P, P, P, P]),
    "dmpc_qp_inspect": (c_int, [P, P, P, P, P, P, P]),
    "dmpc_set_ocps": (c_int, [P, c_int, P, P, P]),
    "dmpc_solve_subset": (c_int, [P, P, c_int, P, P, P, P, P, P, P, P]),
    "dmpc_solve_subset_plain": (c_int, [P, P, c_int, P, P, P, P, P, P, P, P]),
    "dmpc_device_bytes": (ctypes.c_longlong, [P]),
    "dmpc_inspect_offsets": (c_int, [P, P]),
    "dmpc_get_cluster": (c_int, [P, P, P, P]),
    "dmpc_cluster_shape": (c_int, [c_int, c_int, c_int, c_int, c_ll, P, P, P]),
    "dmpc_solve_noalloc": (c_int, [ctypes.POINTER(dmpc_ocp_desc), c_int, ctypes.POINTER(dmpc_options), P,
                                   P, P, P, P, P, P, P, P, P, P]),
    "dmpc_set_solution": (c_int, [P, P, P, P, P, P]),
    "dmpc_set_stream": (c_int, [P, P]),
    "dmpc_set_tiling": (c_int, [P, c_int, c_int]),
    "dmpc_get_tiling": (c_int, [P, P, P, P, P]),
    "dmpc_probe_fp32_peak": (c_int, [P, P]),
    "dmpc_probe_pcg_floor": (c_int, [c_int, P]),
    "dmpc_destroy": (None, [P]),
    "dmpc_last_error": (ctypes.c_char_p, [P]),
    "dmpc_version": (ctypes.c_char_p, []),
}

ERRORS = {0: "DMPC_OK", 1: "DMPC_E_ARG", 2: "DMPC_E_OOM", 3: "DMPC_E_BUDGET", 4: "DMPC_E_CUDA",
          5: "DMPC_E_STATE", 6: "DMPC_E_UNSUPPORTED"}

_lib = None


class DMPCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    """Load libdmpc.so (built by paper_2510_06179_gb300.build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run paper_2510_06179_gb300.build.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(code, handle=None):
    if code != 0:
        msg = load().dmpc_last_error(handle)
        raise DMPCError(code, msg.decode() if msg else "")


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
