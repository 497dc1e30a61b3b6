"""FP64 CPU oracle for the open-system (Lindblad) form of the Tavis-Cummings
evolution.  TEST INFRASTRUCTURE ONLY: imported by the test suite alone; it
shares no code with the GPU library.

The paper writes the quantum master equation (Sec. III.A, Eq. 5) as
    i drho/dt = [H, rho] + i L(rho)          (hbar = 1)
and switches the Lindblad term L off.  This module keeps it on with the
reading used throughout this package: photon leakage from the cavity at rate
kappa,
    L(rho) = kappa (a rho a^dag - 1/2 {a^dag a, rho}).
Leakage lowers the total excitation number k = popcount(s) + p, so the state
lives on the truncated space of all (s, p) with popcount(s) + p <= n (the
closed model is its k = n part, Eqs. 2-4).

Everything here is dense on that space (dimension D = sum_k d_k,
d_k = #{s : popcount(s) <= k}) and written from the definitions:

* ``basis``          the states (s, p), ordered by p, then s.
* ``hamiltonian``    Eq. 4 on the truncated space: omega_c p + omega_a
                     popcount(s) on the diagonal, g_i sqrt(p_e + 1) between
                     (s with atom i excited, p_e) and (s without it, p_e + 1).
* ``annihilation``   a|s, p> = sqrt(p) |s, p - 1>.
* ``liouvillian``    the superoperator of Eq. 5 on row-major vec(rho) (tiny D
                     only); ``exact`` = its exponential (scipy, a library
                     primitive).
* ``damping``        the exact solution of the damping part alone,
                     rho(tau) = sum_m K_m rho K_m^dag,
                     K_m = sqrt((1 - eta)^m / m!) eta^{a^dag a / 2} a^m,
                     eta = e^{-kappa tau} (the bosonic pure-loss channel).
* ``block_propagator`` e^{-iH dt} on the states of one excitation number.
* ``split_step``     one symmetric (Strang) split step of length dt:
                     D_{dt/2}, then rho <- U rho U^dag with U = e^{-iH dt}
                     (from the oracle's Jacobi eigen-decomposition,
                     U = V e^{-i w dt} V^T), then D_{dt/2}.  This is the
                     step the GPU path takes; it differs from ``exact`` by
                     O(dt^3) per step.
* ``observables``    [P_1..P_n, <p>, P(0..n), Tr rho, Tr rho^2, E] with P(m)
                     the probability of m photons.

What pins each function (tests/test_oracle_lindblad.py): ``damping`` against
the exponential of the damping superoperator; ``exact`` against the closed
form of the damped Jaynes-Cummings atom (n = 1); ``split_step`` against
``exact`` at second order in dt and, at kappa = 0, against the closed
oracle's dense step; the dissipator's sign by the excitation balance
d<k>/dt = -kappa <p>; trace, Hermiticity and positivity of every map.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from . import jacobi_eig

COUPLING_BOSONIC = 0
COUPLING_QUBIT_PHOTON = 1


def _popcount(s: int) -> int:
    return bin(s).count("1")


def basis(n: int):
    """States (s, p) with popcount(s) + p <= n, ordered by p then s."""
    out = []
    for p in range(n + 1):
        for s in range(1 << n):
            if _popcount(s) + p <= n:
                out.append((s, p))
    return out


def index(n: int) -> dict:
    return {st: i for i, st in enumerate(basis(n))}


def hamiltonian(n, g, omega_a, omega_c, coupling=COUPLING_BOSONIC) -> np.ndarray:
    """Dense real H of Eq. 4 on the truncated space (atom i = bit n - i)."""
    g = np.asarray(g, dtype=np.float64)
    B = basis(n)
    ix = index(n)
    D = len(B)
    H = np.zeros((D, D))
    for r, (s, p) in enumerate(B):
        H[r, r] = omega_c * p + omega_a * _popcount(s)
        for i in range(1, n + 1):
            bit = 1 << (n - i)
            if s & bit:
                # atom i excited: sigma_i a^dag takes it to (s - bit, p + 1)
                t = (s & ~bit, p + 1)
                if t in ix:
                    h = g[i - 1] if coupling == COUPLING_QUBIT_PHOTON else g[i - 1] * np.sqrt(p + 1.0)
                    H[ix[t], r] = h
                    H[r, ix[t]] = h
    return H


def annihilation(n: int) -> np.ndarray:
    B = basis(n)
    ix = index(n)
    D = len(B)
    a = np.zeros((D, D))
    for r, (s, p) in enumerate(B):
        if p >= 1:
            a[ix[(s, p - 1)], r] = np.sqrt(p)
    return a


def photon_number(n: int) -> np.ndarray:
    return np.array([p for (_, p) in basis(n)], dtype=np.float64)


def excitation_number(n: int) -> np.ndarray:
    return np.array([p + _popcount(s) for (s, p) in basis(n)], dtype=np.float64)


def liouvillian(n, g, omega_a, omega_c, kappa, coupling=COUPLING_BOSONIC, hamiltonian_on=True) -> np.ndarray:
    """Superoperator of Eq. 5 on row-major vec(rho): vec(A rho B) = (A kron B^T) vec(rho)."""
    H = hamiltonian(n, g, omega_a, omega_c, coupling)
    if not hamiltonian_on:
        H = np.zeros_like(H)
    a = annihilation(n)
    D = H.shape[0]
    I = np.eye(D)
    ada = a.T @ a
    L = -1j * (np.kron(H, I) - np.kron(I, H.T))
    L = L + kappa * (np.kron(a, a) - 0.5 * np.kron(ada, I) - 0.5 * np.kron(I, ada.T))
    return L


def exact(n, g, omega_a, omega_c, kappa, t, rho0, coupling=COUPLING_BOSONIC) -> np.ndarray:
    """rho(t) = e^{L t} rho0 by the superoperator exponential (tiny D only)."""
    from scipy.linalg import expm as _expm
    D = rho0.shape[0]
    v = _expm(liouvillian(n, g, omega_a, omega_c, kappa, coupling) * t) @ rho0.reshape(-1)
    return v.reshape(D, D)


def damping(rho, n: int, kappa: float, tau: float) -> np.ndarray:
    """Exact damping over tau: sum_m K_m rho K_m^dag (pure-loss channel)."""
    a = annihilation(n)
    eta = np.exp(-kappa * tau)
    half = np.diag(eta ** (photon_number(n) / 2.0))
    out = np.zeros_like(rho, dtype=np.complex128)
    am = np.eye(a.shape[0])
    for m in range(n + 1):
        K = np.sqrt((1.0 - eta) ** m / factorial(m)) * (half @ am)
        out += K @ rho @ K.conj().T
        am = a @ am
    return out


def propagator(n, g, omega_a, omega_c, dt, coupling=COUPLING_BOSONIC) -> np.ndarray:
    """U = e^{-iH dt} = V e^{-i w dt} V^T from the Jacobi eigen-decomposition."""
    w, V = jacobi_eig(hamiltonian(n, g, omega_a, omega_c, coupling))
    return (V * np.exp(-1j * w * dt)[None, :]) @ V.T


def block_propagator(n, g, omega_a, omega_c, dt, k, coupling=COUPLING_BOSONIC):
    """e^{-iH dt} restricted to the states of excitation number k (H maps that
    set to itself), by Jacobi on the restriction; returns (U_k, indices of
    those states in ``basis`` order)."""
    sel = [i for i, (s, p) in enumerate(basis(n)) if _popcount(s) + p == k]
    H = hamiltonian(n, g, omega_a, omega_c, coupling)[np.ix_(sel, sel)]
    w, V = jacobi_eig(H)
    return (V * np.exp(-1j * w * dt)[None, :]) @ V.T, sel


def split_step(rho, U, n: int, kappa: float, dt: float) -> np.ndarray:
    """D_{dt/2}, then rho <- U rho U^dag, then D_{dt/2}."""
    r = damping(rho, n, kappa, dt / 2.0)
    r = U @ r @ U.conj().T
    return damping(r, n, kappa, dt / 2.0)


def observables(n, g, omega_a, omega_c, rho, coupling=COUPLING_BOSONIC) -> np.ndarray:
    """[P_1..P_n, <p>, P(0..n), Tr rho, Tr rho^2, E] on the truncated space."""
    B = basis(n)
    out = np.zeros(2 * n + 5)
    d = np.real(np.diag(rho))
    for r, (s, p) in enumerate(B):
        for i in range(1, n + 1):
            if s & (1 << (n - i)):
                out[i - 1] += d[r]
        out[n] += p * d[r]
        out[n + 1 + p] += d[r]
        out[2 * n + 2] += d[r]
    out[2 * n + 3] = float(np.sum(np.abs(rho) ** 2))
    out[2 * n + 4] = float(np.real(np.trace(hamiltonian(n, g, omega_a, omega_c, coupling) @ rho)))
    return out


def propagate(n, g, omega_a, omega_c, kappa, dt, steps, rho0, coupling=COUPLING_BOSONIC):
    """`steps` split steps from rho0; returns (rho_T, observable rows for t = 0..T)."""
    U = propagator(n, g, omega_a, omega_c, dt, coupling)
    rho = np.array(rho0, dtype=np.complex128)
    rows = [observables(n, g, omega_a, omega_c, rho, coupling)]
    for _ in range(steps):
        rho = split_step(rho, U, n, kappa, dt)
        rows.append(observables(n, g, omega_a, omega_c, rho, coupling))
    return rho, np.array(rows)


def all_excited(n: int) -> np.ndarray:
    """rho0 = |s = 2^n - 1, p = 0><...| on the truncated space."""
    ix = index(n)
    D = len(ix)
    rho = np.zeros((D, D), dtype=np.complex128)
    j = ix[((1 << n) - 1, 0)]
    rho[j, j] = 1.0
    return rho
