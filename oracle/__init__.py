"""FP64 CPU oracle for Tavis-Cummings unitary evolution (arXiv 2403.06937).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the
CUDA library is checked against.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it.  It shares no code with the GPU
library and never imports it; the GPU library never imports this package.

The arithmetic lives in ``tc_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that no multiply-add is fused behind the reader's
back).  This module only marshals numpy arrays.  Every function states the
passage of the paper it follows; the section and equation numbers are those of
the paper.

Functions and what pins them (tests under ``tests/test_oracle_*.py``):

* ``build_h``           Eq. 4 on the basis of Eq. 2.  Pinned by a hand-expanded
                         n = 2 matrix (golden file) and the n = 1 Rabi form.
* ``state_step`` / ``propagate``
                         Eqs. 6-7 for a pure state by the Taylor series to
                         convergence.  Pinned by the Jaynes-Cummings closed form
                         (n = 1), the qubit-photon product formula (any n), the
                         Dicke tridiagonal, Jacobi diagonalisation, the
                         short-time limit and conservation laws.
* ``expm``              e^{-iHdt} by columns.  Pinned by unitarity, symmetry
                         and the eigen-decomposition.
* ``taylor_fixed``      Eq. 10 as printed (k_max = 10, no shift).  Pinned by the
                         Taylor remainder bound against ``expm``.
* ``dense_step``        Eq. 6 as two dense products.  Pinned by agreement with
                         ``propagate`` on pure states and by invariants.
* ``observables`` / ``observables_pure``
                         Populations, Eq. 13 photon-number probabilities,
                         trace, purity, energy.  Pinned by the closed forms.
* ``jacobi_eig``        Textbook cyclic Jacobi.  Pinned against LAPACK.
* ``dicke_matrix``      Equal-coupling tridiagonal.  Pinned by n = 1, 2 by hand
                         and against the full 2^n propagation.
* ``lindblad`` (module)  The open-system form: Eq. 5 with photon leakage,
                         dense on the truncated space, the exact damping
                         channel and the symmetric split step.  Pinned by the
                         damped Jaynes-Cummings closed form, the damping
                         superoperator's exponential, second-order convergence
                         and the closed-system oracle at kappa = 0
                         (tests/test_oracle_lindblad.py).
* ``tangent_step`` / ``grad_forward``
                         Forward-mode derivative (Van Loan block).  Pinned by
                         central differences of ``propagate`` and exact
                         identities (d/dw_a + d/dw_c = 0; both 0 at resonance).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

COUPLING_BOSONIC = 0
COUPLING_QUBIT_PHOTON = 1
DEFAULT_TOL = 1e-17


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, FP64, no FP contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    """Load a compiled oracle and declare its C signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i, d, L = ctypes.c_int, ctypes.c_double, ctypes.c_long
    sig = {
        "orc_build_h_dense": (None, [i, dp, d, d, i, dp]),
        "orc_state_step": (i, [i, dp, d, d, i, d, d, dp]),
        "orc_observables": (None, [i, dp, d, d, i, dp, dp]),
        "orc_observables_pure": (None, [i, dp, d, d, i, dp, dp]),
        "orc_expm_columns": (i, [i, dp, d, d, i, d, d, dp]),
        "orc_dense_step_rows": (None, [L, dp, dp, dp, L, L]),
        "orc_zgemm": (None, [L, dp, dp, dp]),
        "orc_taylor_fixed": (None, [L, dp, d, i, dp]),
        "orc_jacobi_eig": (i, [i, dp, dp, dp]),
        "orc_dicke_matrix": (None, [i, d, d, d, dp]),
        "orc_tangent_step": (i, [i, dp, d, d, i, i, d, d, dp, dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _g(g) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(g, dtype=np.float64))


def _cplx(a) -> np.ndarray:
    """complex128 C-contiguous array viewed as interleaved doubles."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return a


# --------------------------------------------------------------------------
def build_h(n: int, g, omega_a: float, omega_c: float,
            coupling: int = COUPLING_BOSONIC) -> np.ndarray:
    """Dense real H of Eq. 4 (Sec. II) on the 2^n basis of Eq. 2."""
    g = _g(g)
    assert g.shape == (n,)
    N = 1 << n
    H = np.empty((N, N), dtype=np.float64)
    _load().orc_build_h_dense(n, _p(g), omega_a, omega_c, coupling, _p(H))
    return H


def state_step(n, g, omega_a, omega_c, dt, psi, coupling=COUPLING_BOSONIC,
               tol=DEFAULT_TOL) -> np.ndarray:
    """One step psi <- e^{-iHdt} psi by the Taylor series (Eqs. 6-7)."""
    g = _g(g)
    out = _cplx(psi).copy()
    k = _load().orc_state_step(n, _p(g), omega_a, omega_c, coupling, dt, tol,
                               _p(out.view(np.float64)))
    if k < 0:
        raise RuntimeError("oracle Taylor series did not converge")
    return out


def propagate(n, g, omega_a, omega_c, dt, steps, psi0, coupling=COUPLING_BOSONIC,
              tol=DEFAULT_TOL, observe=True):
    """Pure-state evolution over `steps` steps of size dt (Eq. 6 with rho = psi psi^dag).

    Returns (psi_T, obs) where obs has steps+1 rows (t = 0 and after each
    step) in the layout of ``observables``; obs is None if observe is False.
    """
    g = _g(g)
    lib = _load()
    psi = _cplx(psi0).copy()
    stride = 2 * n + 5
    obs = np.empty((steps + 1, stride)) if observe else None
    row = np.empty(stride)
    if observe:
        lib.orc_observables_pure(n, _p(g), omega_a, omega_c, coupling,
                                 _p(psi.view(np.float64)), _p(row))
        obs[0] = row
    for k in range(steps):
        used = lib.orc_state_step(n, _p(g), omega_a, omega_c, coupling, dt, tol,
                                  _p(psi.view(np.float64)))
        if used < 0:
            raise RuntimeError("oracle Taylor series did not converge")
        if observe:
            lib.orc_observables_pure(n, _p(g), omega_a, omega_c, coupling,
                                     _p(psi.view(np.float64)), _p(row))
            obs[k + 1] = row
    return psi, obs


def expm(n, g, omega_a, omega_c, dt, coupling=COUPLING_BOSONIC, tol=DEFAULT_TOL):
    """U = e^{-iHdt} (Eq. 6), column j = one Taylor step of e_j."""
    g = _g(g)
    N = 1 << n
    U = np.empty((N, N), dtype=np.complex128)
    k = _load().orc_expm_columns(n, _p(g), omega_a, omega_c, coupling, dt, tol,
                                 _p(U.view(np.float64)))
    if k < 0:
        raise RuntimeError("oracle Taylor series did not converge")
    return U


def taylor_fixed(H, dt, kmax=10) -> np.ndarray:
    """Eq. 10 as printed: sum_{k<=kmax} (-iHdt)^k / k! from dense products."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    N = H.shape[0]
    L = np.empty((N, N), dtype=np.complex128)
    _load().orc_taylor_fixed(N, _p(H), dt, kmax, _p(L.view(np.float64)))
    return L


def dense_step(U, rho, rows=None) -> np.ndarray:
    """Eq. 6 as two dense products: rho' = U rho U^dag (rows r0..r1-1 if given)."""
    U = _cplx(U)
    rho = _cplx(rho)
    N = U.shape[0]
    r0, r1 = (0, N) if rows is None else rows
    out = np.empty((r1 - r0, N), dtype=np.complex128)
    _load().orc_dense_step_rows(N, _p(U.view(np.float64)), _p(rho.view(np.float64)),
                                _p(out.view(np.float64)), r0, r1)
    return out


def zgemm(A, B) -> np.ndarray:
    """Plain triple-loop complex product A B."""
    A = _cplx(A)
    B = _cplx(B)
    N = A.shape[0]
    C = np.empty((N, N), dtype=np.complex128)
    _load().orc_zgemm(N, _p(A.view(np.float64)), _p(B.view(np.float64)), _p(C.view(np.float64)))
    return C


def observables(n, g, omega_a, omega_c, rho, coupling=COUPLING_BOSONIC) -> np.ndarray:
    """Observable row [P_1..P_n, <p>, P(0..n), Tr rho, Tr rho^2, E] of a density matrix."""
    g = _g(g)
    rho = _cplx(rho)
    out = np.empty(2 * n + 5)
    _load().orc_observables(n, _p(g), omega_a, omega_c, coupling,
                            _p(rho.view(np.float64)), _p(out))
    return out


def observables_pure(n, g, omega_a, omega_c, psi, coupling=COUPLING_BOSONIC) -> np.ndarray:
    """The same row for rho = psi psi^dag, without forming rho."""
    g = _g(g)
    psi = _cplx(psi)
    out = np.empty(2 * n + 5)
    _load().orc_observables_pure(n, _p(g), omega_a, omega_c, coupling,
                                 _p(psi.view(np.float64)), _p(out))
    return out


def jacobi_eig(A):
    """Cyclic Jacobi: returns (w, V) with A = V diag(w) V^T."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    m = A.shape[0]
    V = np.empty((m, m))
    w = np.empty(m)
    _load().orc_jacobi_eig(m, _p(A), _p(V), _p(w))
    return w, V


def dicke_matrix(n, g, omega_a, omega_c) -> np.ndarray:
    """(n+1) x (n+1) Dicke tridiagonal of Eq. 4 with all g_i = g."""
    D = np.empty((n + 1, n + 1))
    _load().orc_dicke_matrix(n, float(g), omega_a, omega_c, _p(D))
    return D


def evolve_eig(w, V, rho0, t) -> np.ndarray:
    """rho(t) = V e^{-i w t} V^T rho0 V e^{i w t} V^T (no stepping)."""
    ph = np.exp(-1j * w * t)
    Ut = (V * ph[None, :]) @ V.T
    return Ut @ rho0 @ Ut.conj().T


def tangent_step(n, g, omega_a, omega_c, param, dt, dpsi, psi,
                 coupling=COUPLING_BOSONIC, tol=DEFAULT_TOL):
    """One forward-mode step of (dpsi, psi) for parameter `param`."""
    g = _g(g)
    dpsi = _cplx(dpsi).copy()
    psi = _cplx(psi).copy()
    k = _load().orc_tangent_step(n, _p(g), omega_a, omega_c, coupling, param, dt, tol,
                                 _p(dpsi.view(np.float64)), _p(psi.view(np.float64)))
    if k < 0:
        raise RuntimeError("oracle tangent series did not converge")
    return dpsi, psi


def grad_forward(n, g, omega_a, omega_c, dt, steps, psi0, obs_diag,
                 coupling=COUPLING_BOSONIC, params=None) -> np.ndarray:
    """d<O(T)>/d(theta) for O = diag(obs_diag), pure initial state psi0.

    theta = (g_1..g_n, w_a, w_c).  Forward mode: dL = 2 Re <psi_T|O|dpsi_T>.
    """
    params = list(range(n + 2)) if params is None else list(params)
    obs_diag = np.asarray(obs_diag, dtype=np.float64)
    out = np.zeros(n + 2)
    for j in params:
        psi = _cplx(psi0).copy()
        dpsi = np.zeros_like(psi)
        for _ in range(steps):
            dpsi, psi = tangent_step(n, g, omega_a, omega_c, j, dt, dpsi, psi, coupling)
        out[j] = 2.0 * np.real(np.vdot(psi, obs_diag * dpsi))
    return out


def atom_population_operator(n: int, atom: int) -> np.ndarray:
    """diag(l_atom(s)): excited population of atom `atom` (1-based, MSB first)."""
    s = np.arange(1 << n)
    return ((s >> (n - atom)) & 1).astype(np.float64)
