"""ctypes view of libtc's C ABI (include/tc.h).  Marshalling only.

Each function here has the name and argument order of the C entry point.
Pointers are passed as integers (device addresses from torch tensors or host
addresses), streams as integers (cudaStream_t).  A non-zero status raises
TCError with the library's message.  There is no fallback: if the library is
not built, loading raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtc.so")

TC_OK = 0
STATUS_NAMES = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_UNSUPPORTED_DEVICE", 3: "TC_ERR_WORKSPACE",
                4: "TC_ERR_CUDA", 5: "TC_ERR_TIMEOUT", 6: "TC_ERR_NUMERIC"}

TC_FP64, TC_BF16X3, TC_TF32, TC_TF32X3, TC_FP64_OZAKI = 0, 1, 2, 3, 4
TC_COUPLING_BOSONIC, TC_COUPLING_QUBIT_PHOTON = 0, 1
TC_OP_EXPM, TC_OP_EVOLVE, TC_OP_OBSERVABLES, TC_OP_BACKWARD, TC_OP_EVOLVE_HOST, TC_OP_EXPM_MODEL = 1, 2, 4, 8, 16, 32
TC_OP_LINDBLAD = 64
TC_OP_EVOLVE_HOST_PINNED = 128


class TCError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s: %s (%s)" % (where, msg, STATUS_NAMES.get(status, status)))
        self.status = status


class tc_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("g", ctypes.POINTER(ctypes.c_double)), ("omega_a", ctypes.c_double),
                ("omega_c", ctypes.c_double), ("coupling", ctypes.c_int)]


class tc_expm_opts(ctypes.Structure):
    _fields_ = [("taylor_degree", ctypes.c_int), ("squarings", ctypes.c_int), ("shift", ctypes.c_int)]


VP = ctypes.c_void_p
SZ = ctypes.c_size_t
I = ctypes.c_int
D = ctypes.c_double
DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the order of include/tc.h
SIGNATURES = {
    "tc_version": (ctypes.c_char_p, []),
    "tc_last_error": (ctypes.c_char_p, []),
    "tc_device_check": (I, []),
    "tc_workspace_size": (SZ, [I, I, I, I, I]),
    "tc_build_hamiltonian": (I, [ctypes.POINTER(tc_params), VP, VP]),
    "tc_expm": (I, [VP, I, D, ctypes.POINTER(tc_expm_opts), VP, VP, SZ, VP]),
    "tc_expm_model": (I, [ctypes.POINTER(tc_params), D, ctypes.POINTER(tc_expm_opts), VP, VP, SZ, VP]),
    "tc_lindblad_layout": (I, [I, VP, VP, VP]),
    "tc_lindblad_propagators": (I, [ctypes.POINTER(tc_params), D, VP, VP, SZ, VP]),
    "tc_lindblad_evolve": (I, [ctypes.POINTER(tc_params), D, D, VP, VP, I, I, I, VP, VP, SZ, VP]),
    "tc_evolve": (I, [VP, VP, I, I, I, I, ctypes.POINTER(tc_params), VP, VP, SZ, VP]),
    "tc_observables": (I, [VP, I, ctypes.POINTER(tc_params), VP, VP, SZ, VP]),
    "tc_expectation_diag": (I, [VP, I, VP, VP, VP]),
    "tc_observables_noalloc": (I, [VP, I, ctypes.POINTER(tc_params), VP, VP]),
    "tc_evolve_backward": (I, [ctypes.POINTER(tc_params), D, I, VP, VP, I, I, VP, DP, DP, VP, SZ, VP]),
    "tc_evolve_host": (I, [VP, VP, I, I, I, I, ctypes.POINTER(tc_params), VP, VP, SZ, VP]),
    "tc_autotune": (I, [I, I, VP, SZ, VP, ctypes.POINTER(I)]),
    "tc_autotune_lookup": (I, [I, I, ctypes.POINTER(I)]),
    "tc_autotune_set": (I, [I, I, ctypes.POINTER(I)]),
    "tc_batch_autotune": (I, [I, ctypes.POINTER(I), I, VP, SZ, VP, ctypes.POINTER(I)]),
    "tc_batch_autotune_set": (I, [I, ctypes.POINTER(I), I, ctypes.POINTER(I)]),
    "tc_batch_autotune_lookup": (I, [I, ctypes.POINTER(I), I, ctypes.POINTER(I), ctypes.POINTER(I)]),
    "tc_batch_workspace_size": (SZ, [I, ctypes.POINTER(I), I]),
    "tc_batch_evolve": (I, [I, ctypes.POINTER(I), ctypes.POINTER(VP), ctypes.POINTER(VP), I, I, I,
                            ctypes.POINTER(tc_params), ctypes.POINTER(VP), VP, SZ, VP]),
    "tc_launch_count": (ctypes.c_longlong, []),
    "tc_timing_enable": (I, [I]),
    "tc_timing_read": (I, [ctypes.POINTER(ctypes.c_longlong), DP, DP]),
    "tc_phases_enable": (I, [I]),
    "tc_phases_read": (I, [DP, ctypes.c_char_p, SZ, I, ctypes.POINTER(I)]),
    "tc_fault_inject": (I, [I, I, D]),
    "tc_sync_status": (I, [VP]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtc.so (built by paper_2403_06937_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libtc.so is not built (%s); run `python -m paper_2403_06937_gb300.build` "
                           "or __graft_entry__.build() -- there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().tc_last_error().decode()


def check(status: int, where: str) -> None:
    if status != TC_OK:
        raise TCError(status, where, last_error())


def make_params(n: int, g, omega_a: float, omega_c: float, coupling: int = TC_COUPLING_BOSONIC):
    """tc_params plus the ctypes array that keeps g alive."""
    arr = (ctypes.c_double * n)(*[float(x) for x in g])
    p = tc_params(n, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), float(omega_a), float(omega_c),
                  int(coupling))
    p._keep = arr
    return p


def call(name: str, *args) -> int:
    """Call the C entry point `name` and raise on a non-OK status."""
    st = getattr(load(), name)(*args)
    check(st, name)
    return st
