"""Parity of the FP64 CUDA path (through the C ABI) with the CPU oracle.

Tolerances: H is compared bit for bit (same correctly rounded operations);
e^{-iHdt} to 1e-13 max-abs; rho after the stepped evolution to 1e-10 max-abs
(the FP64 target), observables to 1e-10.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_2403_06937_gb300 import build
    build.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    return tc


def _params(tc, n, g, wa, wc, coupling=0):
    return tc.Params(n, list(map(float, g)), wa, wc, coupling)


def _rho_from_states(weights, states):
    return sum(w * np.outer(s, s.conj()) for w, s in zip(weights, states))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
@pytest.mark.parametrize("coupling", [0, 1])
def test_hamiltonian_is_bitwise_equal(tc, oracle, n, coupling):
    g = W.draw_couplings(n, 100 + n)
    H = tc.build_hamiltonian(_params(tc, n, g, 1.002, 0.999, coupling)).cpu().numpy()
    ref = oracle.build_h(n, g, 1.002, 0.999, coupling)
    assert np.array_equal(H, ref)


@pytest.mark.parametrize("n", [1, 3, 5, 6, 7, 9])
def test_expm_matches_oracle(tc, oracle, n):
    g = W.draw_couplings(n, 7) * 3
    p = _params(tc, n, g, 1.002, 1.0)
    H = tc.build_hamiltonian(p)
    U = tc.expm(H, n, 0.05).cpu().numpy()
    ref = oracle.expm(n, g, 1.002, 1.0, 0.05)
    assert np.max(np.abs(U - ref)) < 1e-13
    assert np.array_equal(U, U.T)
    N = 1 << n
    assert np.max(np.abs(U.conj().T @ U - np.eye(N))) < 1e-13


def test_expm_paper_mode_is_eq10(tc, oracle):
    n, dt = 5, 0.1
    g = np.full(n, 0.01)
    p = _params(tc, n, g, 1.0, 1.0)
    H = tc.build_hamiltonian(p)
    U = tc.expm(H, n, dt, taylor_degree=10, squarings=0, shift=False).cpu().numpy()
    L = oracle.taylor_fixed(oracle.build_h(n, g, 1.0, 1.0), dt, 10)
    assert np.max(np.abs(U - (L + L.T) / 2)) < 1e-14
    # and it carries the k_max = 10 truncation error of the paper's scheme
    exact = oracle.expm(n, g, 1.0, 1.0, dt)
    assert np.max(np.abs(U - exact)) > 1e-11


@pytest.mark.parametrize("degree,squarings", [(6, 3), (4, 6), (12, 0)])
def test_expm_forced_plans(tc, oracle, degree, squarings):
    n = 6
    g = W.draw_couplings(n, 3) * 4
    p = _params(tc, n, g, 1.01, 1.0)
    H = tc.build_hamiltonian(p)
    U = tc.expm(H, n, 0.2, taylor_degree=degree, squarings=squarings).cpu().numpy()
    ref = oracle.expm(n, g, 1.01, 1.0, 0.2)
    assert np.max(np.abs(U - ref)) < 1e-12


def test_evolve_n8_workload(tc, oracle):
    """n = 8, dim 256, g = 0.01, dt = 0.1, 100 steps from the all-excited state."""
    cfg = W.config_n8()
    p = _params(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c)
    H = tc.build_hamiltonian(p)
    U = tc.expm(H, cfg.n, cfg.dt)
    rho0 = torch.from_numpy(W.all_excited_rho(cfg.n)).cuda()
    rho, obs = tc.evolve(U, rho0, cfg.n, cfg.steps, "fp64", params=p)
    psi, oobs = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps,
                                 W.all_excited_state(cfg.n))
    rho = rho.cpu().numpy()
    assert np.max(np.abs(rho - np.outer(psi, psi.conj()))) < 1e-10
    assert np.max(np.abs(obs.cpu().numpy() - oobs)) < 1e-10
    assert np.array_equal(rho, rho.conj().T)          # exactly Hermitian by construction


@pytest.mark.parametrize("n,steps", [(1, 30), (4, 25), (6, 20), (7, 9)])
def test_evolve_mixed_state(tc, oracle, n, steps):
    g = W.draw_couplings(n, 40 + n) * 5
    wa, wc, dt = 1.013, 1.0, 0.1
    p = _params(tc, n, g, wa, wc)
    rho0, wts, states = W.random_mixed_state(n, min(3, 1 << n), 5 + n)
    U = tc.expm(tc.build_hamiltonian(p), n, dt)
    rho, obs = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, steps, "fp64", params=p)
    finals = [oracle.propagate(n, g, wa, wc, dt, steps, s, observe=False)[0] for s in states]
    ref = _rho_from_states(wts, finals)
    assert np.max(np.abs(rho.cpu().numpy() - ref)) < 1e-11
    np.testing.assert_allclose(obs.cpu().numpy()[-1], oracle.observables(n, g, wa, wc, ref), atol=1e-11)
    np.testing.assert_allclose(obs.cpu().numpy()[0], oracle.observables(n, g, wa, wc, rho0), atol=1e-12)


def test_zero_steps_leaves_rho(tc):
    n = 3
    p = _params(tc, n, [0.1, 0.2, 0.3], 1.0, 1.0)
    U = tc.expm(tc.build_hamiltonian(p), n, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 1)
    r0 = torch.from_numpy(rho0).cuda()
    rho, obs = tc.evolve(U, r0, n, 0, "fp64", params=p)
    assert torch.equal(rho, r0)
    assert obs.shape == (1, 2 * n + 5)


@pytest.mark.parametrize("n", [2, 7, 9])
def test_observables_match_and_are_deterministic(tc, oracle, n):
    g = W.draw_couplings(n, 9)
    rho0, _, _ = W.random_mixed_state(n, 3, 2)
    p = _params(tc, n, g, 1.05, 0.97)
    r = torch.from_numpy(rho0).cuda()
    a = tc.observables(r, n, p)
    b = tc.observables(r, n, p)
    assert torch.equal(a, b)
    np.testing.assert_allclose(a.cpu().numpy(), oracle.observables(n, g, 1.05, 0.97, rho0), atol=1e-12)
    # without params the energy column is zero
    c = tc.observables(r, n, None).cpu().numpy()
    assert c[-1] == 0.0


def test_renormalisation_restores_the_trace(tc, oracle):
    n = 5
    g = W.draw_couplings(n, 1)
    p = _params(tc, n, g, 1.0, 1.0)
    U = tc.expm(tc.build_hamiltonian(p), n, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 3)
    rho, obs = tc.evolve(U, torch.from_numpy(2.5 * rho0).cuda(), n, 4, "fp64", renorm_every=2, params=p)
    o = obs.cpu().numpy()
    assert abs(o[1, 2 * n + 2] - 2.5) < 1e-12      # not yet renormalised after step 1
    assert abs(o[2, 2 * n + 2] - 1.0) < 1e-14      # renormalised after step 2
    assert abs(o[4, 2 * n + 2] - 1.0) < 1e-14


def test_n12_workload_sampled(tc, oracle):
    """n = 12, dim 4096 (the FP64 at-scale workload): a few steps, sampled entries."""
    cfg = W.config_n12()
    steps = 3
    p = _params(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm(tc.build_hamiltonian(p), cfg.n, cfg.dt)
    rho0 = torch.from_numpy(W.all_excited_rho(cfg.n)).cuda()
    rho, obs = tc.evolve(U, rho0, cfg.n, steps, "fp64", params=p)
    psi, oobs = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, steps, W.all_excited_state(cfg.n))
    rho = rho.cpu().numpy()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, cfg.N, size=(4000, 2))
    idx = np.concatenate([idx, np.array([[cfg.N - 1, cfg.N - 1], [cfg.N - 2, cfg.N - 1], [0, 0]])])
    got = rho[idx[:, 0], idx[:, 1]]
    want = psi[idx[:, 0]] * psi[idx[:, 1]].conj()
    assert np.max(np.abs(got - want)) < 1e-10
    # the heaviest rows/columns (where psi lives) in full
    top = np.argsort(-np.abs(psi))[:64]
    sub = rho[np.ix_(top, top)]
    assert np.max(np.abs(sub - np.outer(psi[top], psi[top].conj()))) < 1e-10
    assert np.max(np.abs(obs.cpu().numpy() - oobs)) < 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["ozaki", "fp64"])
def test_n12_workload_all_200_steps(tc, oracle, precision):
    """The n = 12 FP64 workload over all its 200 steps, in both FP64 product
    forms (DMMA and emulated on the BF16 tensor cores), against the oracle's
    pure-state propagation: every observable row and the final rho (random
    sample plus the block on the heaviest entries) within 1e-10 max-abs."""
    cfg = W.config_n12()
    p = _params(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm(tc.build_hamiltonian(p), cfg.n, cfg.dt)
    rho0 = torch.from_numpy(W.all_excited_rho(cfg.n)).cuda()
    rho, obs = tc.evolve(U, rho0, cfg.n, cfg.steps, precision, params=p)
    tc.sync_status()
    psi, oobs = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps,
                                 W.all_excited_state(cfg.n))
    e_obs = float(np.max(np.abs(obs.cpu().numpy() - oobs)))
    rng = np.random.default_rng(12)
    top = np.argsort(-np.abs(psi))[:64]
    ii = np.concatenate([rng.integers(0, cfg.N, 20000), np.repeat(top, len(top))])
    jj = np.concatenate([rng.integers(0, cfg.N, 20000), np.tile(top, len(top))])
    got = rho[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    e_rho = float(np.max(np.abs(got - psi[ii] * psi[jj].conj())))
    print("n=12, 200 steps, %s: max|obs - oracle| %.2e, max|rho - oracle| %.2e" % (precision, e_obs, e_rho))
    assert e_obs < 1e-10 and e_rho < 1e-10


def test_short_workspace_is_an_error(tc):
    import ctypes
    from paper_2403_06937_gb300 import _abi
    n = 4
    p = _params(tc, n, [0.1] * 4, 1.0, 1.0)
    H = tc.build_hamiltonian(p)
    U = torch.empty((16, 16), dtype=torch.complex128, device="cuda")
    w = torch.empty(512, dtype=torch.uint8, device="cuda")
    st = _abi.load().tc_expm(ctypes.c_void_p(H.data_ptr()), n, 0.1, None, ctypes.c_void_p(U.data_ptr()),
                             ctypes.c_void_p(w.data_ptr()), 512, None)
    assert st == 3
    assert "need" in _abi.last_error()
