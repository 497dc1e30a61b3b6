"""Pins of the open-system oracle (Sec. III.A, Eq. 5 with the Lindblad term of
photon leakage) to results fixed by mathematics, and a check that each pin is
sharp: plausible slips planted in the oracle (on the CPU) break some pin.

Nothing compares the oracle with itself: the damping channel is checked
against the exponential of the damping superoperator and a hand expansion;
the exact evolution against the closed form of the damped Jaynes-Cummings
atom; the split step against the exact evolution at second order in dt and,
at kappa = 0, against the closed-system oracle (Taylor stepping of Eqs. 6-7).
"""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def L(oracle):
    from oracle import lindblad
    return lindblad


def _random_block_rho(L, n, seed):
    """Random density matrix that is block diagonal in the excitation number."""
    rng = np.random.default_rng(seed)
    k = L.excitation_number(n)
    D = len(k)
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    rho = A @ A.conj().T
    rho[k[:, None] != k[None, :]] = 0.0
    return rho / np.trace(rho).real


def _damped_jc_excited(t, g, kappa):
    """|c_e(t)|^2 of the damped Jaynes-Cummings atom at resonance, kappa < 4g."""
    om = math.sqrt(g * g - kappa * kappa / 16.0)
    c = math.exp(-kappa * t / 4.0) * (math.cos(om * t) + kappa / (4.0 * om) * math.sin(om * t))
    return c * c


# ------------------------------------------------------------ the space and a
def pin_basis_and_annihilation(L):
    assert L.basis(1) == [(0, 0), (1, 0), (0, 1)]
    a = L.annihilation(1)
    ref = np.zeros((3, 3))
    ref[0, 2] = 1.0               # a |s=0, p=1> = |s=0, p=0>
    np.testing.assert_array_equal(a, ref)
    for n in (2, 3):
        a = L.annihilation(n)
        np.testing.assert_allclose(a.T @ a, np.diag(L.photon_number(n)), atol=1e-14)
        # dimension: sum over k of #{s : popcount(s) <= k}
        d = sum(sum(math.comb(n, j) for j in range(k + 1)) for k in range(n + 1))
        assert a.shape == (d, d)


def pin_hamiltonian_top_block_is_the_closed_model(L, oracle):
    n = 3
    g = W.draw_couplings(n, 4) * 10
    H = L.hamiltonian(n, g, 1.1, 0.9)
    ix = L.index(n)
    Hc = oracle.build_h(n, g, 1.1, 0.9)
    sel = [ix[(s, n - bin(s).count("1"))] for s in range(1 << n)]
    np.testing.assert_array_equal(H[np.ix_(sel, sel)], Hc)
    # H conserves the excitation number
    k = L.excitation_number(n)
    assert np.all(H[k[:, None] != k[None, :]] == 0.0)


# ------------------------------------------------------------ damping channel
def pin_damping_is_the_superoperator_exponential(L):
    from scipy.linalg import expm
    n, kappa, tau = 2, 0.7, 0.9
    rng = np.random.default_rng(3)
    D = len(L.basis(n))
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    rho = A @ A.conj().T
    Ld = L.liouvillian(n, np.zeros(n), 1.0, 1.0, kappa, hamiltonian_on=False)
    ref = (expm(Ld * tau) @ rho.reshape(-1)).reshape(D, D)
    np.testing.assert_allclose(L.damping(rho, n, kappa, tau), ref, atol=1e-13)


def pin_damping_one_photon_by_hand(L):
    """|g,1> decays to |g,0> with weight 1 - e^{-kappa tau}; the coherence
    <g,0|rho|g,1> shrinks by e^{-kappa tau / 2}."""
    n, kappa, tau = 1, 0.8, 0.6
    ix = L.index(n)
    g0, g1 = ix[(0, 0)], ix[(0, 1)]
    rho = np.zeros((3, 3), dtype=complex)
    rho[g1, g1] = 0.5
    rho[g0, g0] = 0.5
    rho[g0, g1] = rho[g1, g0] = 0.5
    out = L.damping(rho, n, kappa, tau)
    eta = math.exp(-kappa * tau)
    assert abs(out[g1, g1] - 0.5 * eta) < 1e-15
    assert abs(out[g0, g0] - (0.5 + 0.5 * (1 - eta))) < 1e-15
    assert abs(out[g0, g1] - 0.5 * math.sqrt(eta)) < 1e-15


def pin_damping_is_cptp(L):
    n, kappa, tau = 3, 1.3, 0.4
    rho = _random_block_rho(L, n, 5)
    out = L.damping(rho, n, kappa, tau)
    assert abs(np.trace(out) - 1.0) < 1e-14
    np.testing.assert_allclose(out, out.conj().T, atol=1e-15)
    assert np.min(np.linalg.eigvalsh(out)) > -1e-14


# ------------------------------------------------------------ exact evolution
def pin_damped_jaynes_cummings(L):
    g, kappa = 0.3, 0.4
    ix = L.index(1)
    e0 = ix[(1, 0)]
    rho0 = np.zeros((3, 3), dtype=complex)
    rho0[e0, e0] = 1.0
    for t in (0.5, 2.0, 7.0):
        r = L.exact(1, [g], 1.0, 1.0, kappa, t, rho0)
        assert abs(r[e0, e0].real - _damped_jc_excited(t, g, kappa)) < 1e-12
        assert abs(np.trace(r) - 1.0) < 1e-12


def pin_excitation_balance(L):
    """d Tr(K rho)/dt = -kappa Tr(a^dag a rho): H conserves K, leakage lowers it."""
    n, kappa = 2, 0.9
    g = W.draw_couplings(n, 2) * 20
    Lv = L.liouvillian(n, g, 1.02, 0.97, kappa)
    rho = _random_block_rho(L, n, 7)
    D = rho.shape[0]
    drho = (Lv @ rho.reshape(-1)).reshape(D, D)
    lhs = np.sum(L.excitation_number(n) * np.real(np.diag(drho)))
    rhs = -kappa * np.sum(L.photon_number(n) * np.real(np.diag(rho)))
    assert abs(lhs - rhs) < 1e-13


# ------------------------------------------------------------ the split step
def pin_split_step_is_second_order(L):
    n, kappa, T = 2, 0.5, 1.0
    g = W.draw_couplings(n, 8) * 40
    rho0 = _random_block_rho(L, n, 9)
    ref = L.exact(n, g, 1.01, 1.0, kappa, T, rho0)
    errs = []
    for steps in (8, 16, 32):
        r, _ = L.propagate(n, g, 1.01, 1.0, kappa, T / steps, steps, rho0)
        errs.append(np.max(np.abs(r - ref)))
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5, errs


def pin_kappa_zero_is_the_closed_oracle(L, oracle):
    n, dt, steps = 4, 0.1, 20
    g = W.draw_couplings(n, 6) * 5
    rho, rows = L.propagate(n, g, 1.002, 1.0, 0.0, dt, steps, L.all_excited(n))
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[-1] = 1.0
    psi, obs = oracle.propagate(n, g, 1.002, 1.0, dt, steps, psi0)
    ix = L.index(n)
    sel = [ix[(s, n - bin(s).count("1"))] for s in range(1 << n)]
    np.testing.assert_allclose(rho[np.ix_(sel, sel)], np.outer(psi, psi.conj()), atol=1e-12)
    rest = np.ones(rho.shape[0], bool)
    rest[sel] = False
    assert np.max(np.abs(rho[rest])) == 0.0
    np.testing.assert_allclose(rows, obs, atol=1e-12)


def pin_split_step_keeps_blocks_and_trace(L):
    n, kappa, dt = 3, 0.6, 0.2
    g = W.draw_couplings(n, 10) * 30
    rho0 = _random_block_rho(L, n, 11)
    rho, rows = L.propagate(n, g, 1.0, 1.0, kappa, dt, 10, rho0)
    k = L.excitation_number(n)
    assert np.max(np.abs(rho[k[:, None] != k[None, :]])) < 1e-14
    np.testing.assert_allclose(rows[:, 2 * n + 2], 1.0, atol=1e-13)
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-14
    # photons leak: the mean excitation number never grows
    kk = [np.sum(k * np.real(np.diag(r))) for r in [rho0, rho]]
    assert kk[1] < kk[0]


def pin_block_propagator_is_a_block_of_the_full_one(L):
    n, dt = 4, 0.3
    g = W.draw_couplings(n, 12) * 30
    U = L.propagator(n, g, 1.01, 0.99, dt)
    for k in range(n + 1):
        Uk, sel = L.block_propagator(n, g, 1.01, 0.99, dt, k)
        np.testing.assert_allclose(Uk, U[np.ix_(sel, sel)], atol=1e-13)


PINS = [pin_block_propagator_is_a_block_of_the_full_one, pin_basis_and_annihilation, pin_damping_is_the_superoperator_exponential, pin_damping_one_photon_by_hand,
        pin_damping_is_cptp, pin_damped_jaynes_cummings, pin_excitation_balance, pin_split_step_is_second_order,
        pin_split_step_keeps_blocks_and_trace]
PINS_WITH_ORACLE = [pin_hamiltonian_top_block_is_the_closed_model, pin_kappa_zero_is_the_closed_oracle]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(L, pin):
    pin(L)


@pytest.mark.parametrize("pin", PINS_WITH_ORACLE, ids=lambda f: f.__name__)
def test_pin_with_closed_oracle(L, oracle, pin):
    pin(L, oracle)


# ------------------------------------------------------------ sharpness
def _mutants(L):
    from math import factorial

    def damping_no_factorial(rho, n, kappa, tau):
        a = L.annihilation(n)
        eta = np.exp(-kappa * tau)
        half = np.diag(eta ** (L.photon_number(n) / 2.0))
        out = np.zeros_like(rho, dtype=np.complex128)
        am = np.eye(a.shape[0])
        for m in range(n + 1):
            K = np.sqrt((1.0 - eta) ** m) * (half @ am)
            out += K @ rho @ K.conj().T
            am = a @ am
        return out

    def damping_full_eta(rho, n, kappa, tau):
        a = L.annihilation(n)
        eta = np.exp(-kappa * tau)
        half = np.diag(eta ** L.photon_number(n))
        out = np.zeros_like(rho, dtype=np.complex128)
        am = np.eye(a.shape[0])
        for m in range(n + 1):
            K = np.sqrt((1.0 - eta) ** m / factorial(m)) * (half @ am)
            out += K @ rho @ K.conj().T
            am = a @ am
        return out

    def split_full_dt(rho, U, n, kappa, dt):
        r = L.damping(rho, n, kappa, dt)
        r = U @ r @ U.conj().T
        return L.damping(r, n, kappa, dt)

    def split_lie(rho, U, n, kappa, dt):
        return L.damping(U @ rho @ U.conj().T, n, kappa, dt)

    def annihilation_sqrt_p_plus_1(n):
        B = L.basis(n)
        ix = L.index(n)
        a = np.zeros((len(B), len(B)))
        for r, (s, p) in enumerate(B):
            if p >= 1:
                a[ix[(s, p - 1)], r] = np.sqrt(p + 1)
        return a

    def liouvillian_sign(n, g, omega_a, omega_c, kappa, coupling=0, hamiltonian_on=True):
        return L.__dict__["_orig_liouvillian"](n, g, omega_a, omega_c, -kappa, coupling, hamiltonian_on)

    return {"damping_no_factorial": ("damping", damping_no_factorial),
            "damping_full_eta": ("damping", damping_full_eta),
            "split_full_dt": ("split_step", split_full_dt),
            "split_first_order": ("split_step", split_lie),
            "annihilation_sqrt_p_plus_1": ("annihilation", annihilation_sqrt_p_plus_1),
            "liouvillian_dissipator_sign": ("liouvillian", liouvillian_sign)}


@pytest.mark.parametrize("name", ["damping_no_factorial", "damping_full_eta", "split_full_dt", "split_first_order",
                                  "annihilation_sqrt_p_plus_1", "liouvillian_dissipator_sign"])
def test_planted_mistake_is_caught(L, oracle, monkeypatch, name):
    monkeypatch.setitem(L.__dict__, "_orig_liouvillian", L.liouvillian)
    attr, fn = _mutants(L)[name]
    monkeypatch.setattr(L, attr, fn)
    failed = []
    for pin in PINS:
        try:
            pin(L)
        except AssertionError:
            failed.append(pin.__name__)
    for pin in PINS_WITH_ORACLE:
        try:
            pin(L, oracle)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "mutant %s survived every pin" % name
