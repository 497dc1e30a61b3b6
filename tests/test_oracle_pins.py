"""Pins of the CPU oracle to results fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check is a closed form,
a hand expansion, a library routine on a special case, an exact identity or
an independent algorithm (diagonalisation versus Taylor stepping).  A wrong
sign of i, a dropped sqrt(p+1), a swapped atom index or a transposed
operand in the oracle breaks at least one of them.
"""
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rabi_excited(t, g, delta):
    """Jaynes-Cummings, one atom from |e, 0 photons>: excited population."""
    om2 = 4 * g * g + delta * delta
    return 1.0 - (4 * g * g / om2) * np.sin(np.sqrt(om2) * t / 2.0) ** 2


def _expm_2x2_closed(a, b, g, t):
    """exp(-i t [[a, g], [g, b]]) by the closed form of a 2x2 Hermitian matrix."""
    m = 0.5 * (a + b)
    om = math.sqrt((a - b) ** 2 + 4 * g * g)
    K = np.array([[a - m, g], [g, b - m]])
    c, s = math.cos(om * t / 2), math.sin(om * t / 2)
    return np.exp(-1j * m * t) * (c * np.eye(2) - 1j * s * (2.0 / om) * K)


# ------------------------------------------------------------------ Eq. 4
def test_h_n2_matches_hand_expansion(oracle):
    g1, g2, wa, wc = 0.3, 0.7, 1.25, 0.5
    H = oracle.build_h(2, [g1, g2], wa, wc)
    ref = np.zeros((4, 4))
    env = {"g1": g1, "g2": g2, "wa": wa, "wc": wc, "sqrt": math.sqrt}
    with open(os.path.join(GOLDEN, "h_n2_bosonic.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            r, c, expr = line.split(None, 2)
            ref[int(r), int(c)] = eval(expr, {"__builtins__": {}}, env)
    np.testing.assert_allclose(H, ref, rtol=0, atol=1e-15)


def test_h_n1_is_jaynes_cummings(oracle):
    H = oracle.build_h(1, [0.2], 1.5, 0.75)
    # s=0: atom relaxed, one photon (w_c); s=1: atom excited, no photon (w_a)
    np.testing.assert_array_equal(H, np.array([[0.75, 0.2], [0.2, 1.5]]))


@pytest.mark.parametrize("n", [3, 6])
def test_h_structure(oracle, n):
    g = W.draw_couplings(n, 5)
    H = oracle.build_h(n, g, 1.1, 0.9)
    N = 1 << n
    assert np.array_equal(H, H.T)
    nz = np.argwhere(H != 0)
    off = [(a, b) for a, b in nz if a != b]
    assert len(off) == n * N  # n*N/2 symmetric pairs
    for a, b in off:
        assert bin(int(a) ^ int(b)).count("1") == 1
    # qubit-photon reading drops the sqrt(p+1)
    Hq = oracle.build_h(n, g, 1.1, 0.9, coupling=oracle.COUPLING_QUBIT_PHOTON)
    s = np.arange(N)
    for a, b in off[:50]:
        e = max(a, b)  # excited side has the bit set
        p = n - bin(int(e)).count("1")
        i = n - int(math.log2(int(a) ^ int(b)))  # atom index of the flipped bit
        assert H[a, b] == pytest.approx(g[i - 1] * math.sqrt(p + 1), rel=1e-15)
        assert Hq[a, b] == pytest.approx(g[i - 1], rel=1e-15)
    assert np.array_equal(np.diag(H), np.diag(Hq))
    del s


# ----------------------------------------------------- Eqs. 6-8, closed forms
@pytest.mark.parametrize("delta", [0.0, 0.02, -0.37])
def test_jaynes_cummings_rabi(oracle, delta):
    g, wc = 0.05, 1.0
    wa = wc + delta
    dt, steps = 0.25, 80
    psi0 = W.all_excited_state(1)
    _, obs = oracle.propagate(1, [g], wa, wc, dt, steps, psi0)
    t = dt * np.arange(steps + 1)
    np.testing.assert_allclose(obs[:, 0], _rabi_excited(t, g, delta), rtol=0, atol=1e-13)
    # photon number + excited population = 1 (closed system, Eq. 2)
    np.testing.assert_allclose(obs[:, 1] + obs[:, 0], 1.0, atol=1e-14)


def test_jaynes_cummings_full_state_pins_the_sign_of_i(oracle):
    # populations are even in t; the phases of psi(t) are not.
    g, wa, wc, dt, steps = 0.3, 1.7, 0.4, 0.05, 40
    psi, _ = oracle.propagate(1, [g], wa, wc, dt, steps, W.all_excited_state(1))
    # basis order (s=0: relaxed+photon, diag wc; s=1: excited, diag wa)
    Ut = _expm_2x2_closed(wc, wa, g, dt * steps)
    np.testing.assert_allclose(psi, Ut @ np.array([0, 1], dtype=complex), atol=1e-13)
    U = oracle.expm(1, [g], wa, wc, dt)
    np.testing.assert_allclose(U, _expm_2x2_closed(wc, wa, g, dt), atol=1e-15)


@pytest.mark.parametrize("n", [3, 7])
def test_qubit_photon_reading_factorises(oracle, n):
    """Eq. 1 reading: H is a sum of commuting single-atom terms -> independent JC atoms."""
    g = W.draw_couplings(n, 11) * 10
    wc, wa = 1.0, 1.013
    dt, steps = 0.2, 60
    _, obs = oracle.propagate(n, g, wa, wc, dt, steps, W.all_excited_state(n),
                              coupling=oracle.COUPLING_QUBIT_PHOTON)
    t = dt * np.arange(steps + 1)
    q = np.stack([_rabi_excited(t, gi, wa - wc) for gi in g], axis=1)  # P_i(t)
    np.testing.assert_allclose(obs[:, :n], q, atol=1e-12)
    # P(m): Poisson-binomial probability that exactly n-m atoms are excited
    for row in range(0, steps + 1, 7):
        dist = np.array([1.0])
        for qi in q[row]:
            dist = np.convolve(dist, [1 - qi, qi])  # dist[k] = P(k excited)
        Pm = dist[::-1]                              # m = n - k free photons
        np.testing.assert_allclose(obs[row, n + 1:2 * n + 2], Pm, atol=1e-12)


def test_dicke_matrix_by_hand(oracle):
    g, wa, wc = 0.1, 1.3, 0.8
    np.testing.assert_allclose(oracle.dicke_matrix(1, g, wa, wc), [[wa, g], [g, wc]], atol=0)
    D2 = oracle.dicke_matrix(2, g, wa, wc)
    ref = np.array([[2 * wa, math.sqrt(2) * g, 0],
                    [math.sqrt(2) * g, wa + wc, 2 * g],
                    [0, 2 * g, 2 * wc]])
    np.testing.assert_allclose(D2, ref, atol=1e-16)


@pytest.mark.parametrize("n", [2, 5, 8])
def test_dicke_tridiagonal_matches_full_space(oracle, n):
    """Equal couplings: the full 2^n evolution stays in the symmetric subspace."""
    g, wa, wc, dt, steps = 0.07, 1.004, 1.0, 0.3, 40
    _, obs = oracle.propagate(n, np.full(n, g), wa, wc, dt, steps, W.all_excited_state(n))
    D = oracle.dicke_matrix(n, g, wa, wc)
    w, V = oracle.jacobi_eig(D)
    e0 = np.zeros(n + 1)
    e0[0] = 1.0
    for k in range(0, steps + 1, 5):
        amp = (V * np.exp(-1j * w * dt * k)[None, :]) @ (V.T @ e0)
        Pm = np.abs(amp) ** 2
        np.testing.assert_allclose(obs[k, n + 1:2 * n + 2], Pm, atol=1e-12)
        pmean = float(np.dot(np.arange(n + 1), Pm))
        np.testing.assert_allclose(obs[k, :n], (n - pmean) / n, atol=1e-12)


def test_jacobi_against_lapack(oracle):
    rng = np.random.default_rng(3)
    for m in (1, 2, 5, 16, 40):
        A = rng.standard_normal((m, m))
        A = A + A.T
        w, V = oracle.jacobi_eig(A)
        np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12)
        np.testing.assert_allclose((V * w[None, :]) @ V.T, A, atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-13)


@pytest.mark.parametrize("n", [4, 6])
def test_taylor_stepping_matches_diagonalisation(oracle, n):
    g = W.draw_couplings(n, 7) * 5
    wa, wc, dt, steps = 1.01, 1.0, 0.1, 30
    H = oracle.build_h(n, g, wa, wc)
    w, V = oracle.jacobi_eig(H)
    rho0, wts, states = W.random_mixed_state(n, 3, 9)
    rho_t = oracle.evolve_eig(w, V, rho0, dt * steps)
    acc = np.zeros_like(rho0)
    for wr, psi in zip(wts, states):
        pt, _ = oracle.propagate(n, g, wa, wc, dt, steps, psi, observe=False)
        acc += wr * np.outer(pt, pt.conj())
    np.testing.assert_allclose(acc, rho_t, atol=1e-12)
    U = oracle.expm(n, g, wa, wc, dt)
    np.testing.assert_allclose(U, (V * np.exp(-1j * w * dt)[None, :]) @ V.T, atol=1e-13)


def test_short_time_photon_growth(oracle):
    """From all-excited, <p>(t) = (sum g_i^2) t^2 + O(t^4)."""
    n = 6
    g = W.draw_couplings(n, 4)
    tau = 1e-2
    psi = oracle.state_step(n, g, 1.003, 1.0, tau, W.all_excited_state(n))
    pm = oracle.observables_pure(n, g, 1.003, 1.0, psi)[n]
    np.testing.assert_allclose(pm / tau ** 2, np.sum(g ** 2), rtol=1e-4)


def test_invariants_of_pure_evolution(oracle):
    cfg = W.config_n8()
    n = 6
    g = W.draw_couplings(n, 21)
    wa, wc = 1.002, 1.0
    _, obs = oracle.propagate(n, g, wa, wc, cfg.dt, 60, W.all_excited_state(n))
    np.testing.assert_allclose(obs[:, 2 * n + 2], 1.0, atol=1e-13)           # Tr rho
    np.testing.assert_allclose(obs[:, 2 * n + 3], 1.0, atol=1e-13)           # purity
    np.testing.assert_allclose(obs[:, 2 * n + 4], n * wa, atol=1e-12)        # energy
    np.testing.assert_allclose(obs[:, n] + obs[:, :n].sum(1), n, atol=1e-12) # <p> + sum P_i
    np.testing.assert_allclose(obs[:, n + 1:2 * n + 2].sum(1), 1.0, atol=1e-13)


# ---------------------------------------------------------- U and Eq. 10
def test_expm_unitary_and_symmetric(oracle):
    n = 7
    U = oracle.expm(n, W.draw_couplings(n, 1), 1.002, 1.0, 0.05)
    N = 1 << n
    np.testing.assert_allclose(U.conj().T @ U, np.eye(N), atol=1e-14)
    np.testing.assert_allclose(U, U.T, atol=1e-15)


def test_paper_taylor_k10_has_the_predicted_remainder(oracle):
    """Eq. 10 truncates at k_max = 10: L - e^{-iHdt} ~= -(-iHdt)^11/11! to leading order."""
    n, dt = 5, 0.1
    g = np.full(n, 0.01)
    H = oracle.build_h(n, g, 1.0, 1.0)
    L = oracle.taylor_fixed(H, dt, 10)
    U = oracle.expm(n, g, 1.0, 1.0, dt)
    A = -1j * H * dt
    A11 = np.linalg.matrix_power(A, 11) / math.factorial(11)
    err = L - U
    assert np.max(np.abs(err + A11)) <= 0.2 * np.max(np.abs(A11))
    assert np.max(np.abs(A11)) > 1e-11  # ~ ||Hdt||^11/11!, visible in FP64
    # the full series (k_max large) agrees with the converged columns
    np.testing.assert_allclose(oracle.taylor_fixed(H, dt, 25), U, atol=2e-15)


# ---------------------------------------------------------- Eq. 6 dense
def test_dense_step_matches_state_propagation(oracle):
    n = 5
    g = W.draw_couplings(n, 2) * 4
    U = oracle.expm(n, g, 1.01, 1.0, 0.1)
    psi = W.random_pure_state(n, 5)
    rho = np.outer(psi, psi.conj())
    r1 = oracle.dense_step(U, rho)
    p1 = oracle.state_step(n, g, 1.01, 1.0, 0.1, psi)
    np.testing.assert_allclose(r1, np.outer(p1, p1.conj()), atol=1e-14)
    # a row range is the same rows
    np.testing.assert_allclose(oracle.dense_step(U, rho, rows=(3, 9)), r1[3:9], atol=0)


def test_dense_step_general_unitary(oracle):
    """With a non-symmetric unitary the two products must keep their operand order."""
    rng = np.random.default_rng(12)
    Z = rng.standard_normal((24, 24)) + 1j * rng.standard_normal((24, 24))
    Q, _ = np.linalg.qr(Z)
    assert np.max(np.abs(Q - Q.T)) > 0.1
    rho, _, _ = W.random_mixed_state(3, 2, 4)
    rho = np.kron(rho, np.eye(3) / 3.0)
    np.testing.assert_allclose(oracle.dense_step(Q, rho), Q @ rho @ Q.conj().T, atol=1e-14)


def test_dense_step_mixed_invariants(oracle):
    n = 5
    g = W.draw_couplings(n, 2) * 4
    U = oracle.expm(n, g, 1.01, 1.0, 0.1)
    rho, _, _ = W.random_mixed_state(n, 4, 8)
    r1 = oracle.dense_step(U, rho)
    np.testing.assert_allclose(np.trace(r1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.sum(np.abs(r1) ** 2), np.sum(np.abs(rho) ** 2), atol=1e-14)
    np.testing.assert_allclose(r1, r1.conj().T, atol=1e-15)


def test_zgemm_is_a_plain_product(oracle):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((17, 17)) + 1j * rng.standard_normal((17, 17))
    B = rng.standard_normal((17, 17)) + 1j * rng.standard_normal((17, 17))
    np.testing.assert_allclose(oracle.zgemm(A, B), A @ B, atol=1e-13)


# ---------------------------------------------------------- observables
def test_observables_hand_n2(oracle):
    g, wa, wc = [0.3, 0.7], 1.25, 0.5
    d = np.array([0.1, 0.2, 0.3, 0.4])
    rho = np.diag(d).astype(complex)
    rho[3, 1] = rho[1, 3] = 0.05     # coupled pair (atom 1 flip, H = g1)
    rho[2, 1] = 0.01 + 0.02j         # uncoupled pair
    rho[1, 2] = 0.01 - 0.02j
    o = oracle.observables(2, g, wa, wc, rho)
    # P_1: s with l_1 = 1 -> s in {2, 3};  P_2: s in {1, 3}
    assert o[0] == pytest.approx(0.7)
    assert o[1] == pytest.approx(0.6)
    assert o[2] == pytest.approx(0.1 * 2 + 0.2 + 0.3)          # <p>
    np.testing.assert_allclose(o[3:6], [0.4, 0.5, 0.1])       # P(0), P(1), P(2)
    assert o[6] == pytest.approx(1.0)
    assert o[7] == pytest.approx(np.sum(np.abs(rho) ** 2))
    E = 0.1 * 2 * wc + (0.2 + 0.3) * (wc + wa) + 0.4 * 2 * wa + 2 * 0.3 * 0.05
    assert o[8] == pytest.approx(E)


def test_observables_pure_equals_dense(oracle):
    n = 6
    g = W.draw_couplings(n, 3)
    psi = W.random_pure_state(n, 1)
    a = oracle.observables(n, g, 1.02, 0.98, np.outer(psi, psi.conj()))
    b = oracle.observables_pure(n, g, 1.02, 0.98, psi)
    np.testing.assert_allclose(a, b, atol=1e-13)


# ---------------------------------------------------------- gradients
def test_forward_gradient_matches_central_differences(oracle):
    n, dt, steps = 4, 0.3, 12
    g = W.draw_couplings(n, 1) * 8
    wa, wc = 1.02, 1.0
    O = oracle.atom_population_operator(n, 1)
    psi0 = W.all_excited_state(n)
    grad = oracle.grad_forward(n, g, wa, wc, dt, steps, psi0, O)

    def loss(g_, wa_, wc_):
        p, _ = oracle.propagate(n, g_, wa_, wc_, dt, steps, psi0, observe=False)
        return float(np.real(np.vdot(p, O * p)))

    h = 1e-6
    fd = np.zeros(n + 2)
    for j in range(n):
        gp, gm = g.copy(), g.copy()
        gp[j] += h
        gm[j] -= h
        fd[j] = (loss(gp, wa, wc) - loss(gm, wa, wc)) / (2 * h)
    fd[n] = (loss(g, wa + h, wc) - loss(g, wa - h, wc)) / (2 * h)
    fd[n + 1] = (loss(g, wa, wc + h) - loss(g, wa, wc - h)) / (2 * h)
    scale = np.max(np.abs(fd))
    np.testing.assert_allclose(grad, fd, atol=1e-6 * scale)


def test_gradient_identities(oracle):
    n, dt, steps = 4, 0.3, 10
    g = W.draw_couplings(n, 6) * 8
    O = oracle.atom_population_operator(n, 2)
    psi0 = W.all_excited_state(n)
    gd = oracle.grad_forward(n, g, 1.05, 1.0, dt, steps, psi0, O)
    # dH/dw_a + dH/dw_c = n I commutes with everything
    assert abs(gd[n] + gd[n + 1]) <= 1e-12 * max(1.0, abs(gd[n]))
    assert abs(gd[n]) > 1e-6
    gr = oracle.grad_forward(n, g, 1.0, 1.0, dt, steps, psi0, O)
    # at resonance populations are even in the detuning
    assert abs(gr[n]) < 1e-12 and abs(gr[n + 1]) < 1e-12


def test_fig3_claims_hold_under_the_qubit_photon_reading(oracle):
    """The qualitative claims of Sec. IV (Figs. 3-4) -- P(0) falls from 1, the
    P(m) peak in the order m = 1..n, the curves are symmetric about n/2 --
    are exact for equal couplings at resonance under the Eq. 1 (qubit-photon)
    reading, where the atoms are independent: with s = sin^2(g t),
    P(m)(t) = C(n, m) s^m (1 - s)^(n - m), which peaks at s = m / n, and
    P(m)(t) = P(n - m)(pi / (2 g) - t).  n = 8 from the all-excited state (the
    Fig. 3 workload), over a quarter Rabi period on a grid that hits its end."""
    n, g = 8, 0.01
    K = 300
    T = math.pi / (2 * g)
    dt = T / K
    _, obs = oracle.propagate(n, [g] * n, 1.0, 1.0, dt, K, W.all_excited_state(n),
                              coupling=oracle.COUPLING_QUBIT_PHOTON)
    P = obs[:, n + 1:2 * n + 2]            # P(m), m = 0..n, at t = k dt
    assert abs(P[0, 0] - 1.0) < 1e-14 and np.all(np.diff(P[:, 0]) < 1e-15)   # falls from 1 to ~0
    peaks = [int(np.argmax(P[:, m])) for m in range(1, n + 1)]
    assert all(a < b for a, b in zip(peaks, peaks[1:]))
    for m, k in zip(range(1, n + 1), peaks):
        assert abs(k - math.asin(math.sqrt(m / n)) / g / dt) <= 1.0
    for m in range(n + 1):
        np.testing.assert_allclose(P[:, m], P[::-1, n - m], atol=1e-12)
