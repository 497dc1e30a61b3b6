"""Reverse-mode gradient (tc_evolve_backward) against independent checks.

* The oracle's forward-mode tangent (Van Loan block propagation, a different
  algorithm: no adjoint, no Frechet derivative, no checkpoints).
* Central finite differences with h = 1e-6 (of the GPU FP64 forward at small
  n, of the oracle forward at the n = 11 workload).  Their error floor is
  ~eps |L| / h ~ 1e-10 absolute plus h^2 |L'''| terms.
* Exact identities: dL/dw_a + dL/dw_c = 0 (dH/dw_a + dH/dw_c = n I), and both
  vanish at resonance (populations are even in the detuning).

Tolerance: |adj_j - ref_j| <= 1e-6 max(|ref_j|, max_j |ref_j|) for finite
differences (the stated target) and 1e-9 of max|ref| against the oracle
tangent (both FP64).
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


def _gpu_grad(tc, n, g, wa, wc, dt, steps, ckpt, atom, psi0=None, coupling=0, precision="fp64"):
    p = tc.Params(n, list(map(float, g)), wa, wc, coupling)
    U = tc.expm(tc.build_hamiltonian(p), n, dt)
    N = 1 << n
    if psi0 is None:
        rho0 = torch.from_numpy(W.all_excited_rho(n)).cuda()
    else:
        rho0 = torch.from_numpy(np.outer(psi0, psi0.conj())).cuda()
    s = np.arange(N)
    O = torch.from_numpy(((s >> (n - atom)) & 1).astype(np.float64)).cuda()
    grad, loss = tc.evolve_backward(p, dt, steps, rho0, U, O, ckpt_every=ckpt, precision=precision)
    return grad.numpy(), loss


def _gpu_loss(tc, n, g, wa, wc, dt, steps, atom):
    p = tc.Params(n, list(map(float, g)), wa, wc)
    U = tc.expm(tc.build_hamiltonian(p), n, dt)
    rho0 = torch.from_numpy(W.all_excited_rho(n)).cuda()
    _, obs = tc.evolve(U, rho0, n, steps, "fp64", params=p)
    return float(obs[-1, atom - 1].item())


@pytest.mark.parametrize("n,steps,ckpt", [(1, 7, 3), (3, 12, 5), (5, 12, 4), (6, 9, 9)])
def test_adjoint_matches_oracle_tangent(tc, oracle, n, steps, ckpt):
    g = W.draw_couplings(n, 10 + n) * 8
    wa, wc, dt = 1.03, 1.0, 0.3
    grad, loss = _gpu_grad(tc, n, g, wa, wc, dt, steps, ckpt, atom=1)
    O = oracle.atom_population_operator(n, 1)
    ref = oracle.grad_forward(n, g, wa, wc, dt, steps, W.all_excited_state(n), O)
    assert np.max(np.abs(grad - ref)) <= 1e-9 * max(np.max(np.abs(ref)), 1e-12)
    psi, obs = oracle.propagate(n, g, wa, wc, dt, steps, W.all_excited_state(n))
    assert abs(loss - obs[-1, 0]) < 1e-12


def test_adjoint_with_mixed_initial_state_and_other_atom(tc, oracle):
    n, steps, dt = 4, 10, 0.25
    g = W.draw_couplings(n, 3) * 8
    psi0 = W.random_pure_state(n, 8)
    grad, _ = _gpu_grad(tc, n, g, 1.02, 1.0, dt, steps, 3, atom=3, psi0=psi0)
    ref = oracle.grad_forward(n, g, 1.02, 1.0, dt, steps, psi0, oracle.atom_population_operator(n, 3))
    assert np.max(np.abs(grad - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_adjoint_matches_central_differences_of_gpu_forward(tc):
    n, steps, dt = 5, 15, 0.3
    g = W.draw_couplings(n, 2) * 8
    wa, wc = 1.02, 1.0
    grad, _ = _gpu_grad(tc, n, g, wa, wc, dt, steps, 4, atom=1)
    h = 1e-6
    fd = np.zeros(n + 2)
    for j in range(n):
        gp, gm = g.copy(), g.copy()
        gp[j] += h
        gm[j] -= h
        fd[j] = (_gpu_loss(tc, n, gp, wa, wc, dt, steps, 1) - _gpu_loss(tc, n, gm, wa, wc, dt, steps, 1)) / (2 * h)
    fd[n] = (_gpu_loss(tc, n, g, wa + h, wc, dt, steps, 1) - _gpu_loss(tc, n, g, wa - h, wc, dt, steps, 1)) / (2 * h)
    fd[n + 1] = (_gpu_loss(tc, n, g, wa, wc + h, dt, steps, 1) - _gpu_loss(tc, n, g, wa, wc - h, dt, steps, 1)) / (2 * h)
    tol = 1e-6 * np.maximum(np.abs(fd), np.max(np.abs(fd)))
    assert np.all(np.abs(grad - fd) <= tol), (grad, fd)


def test_exact_identities(tc):
    n, steps, dt = 5, 10, 0.3
    g = W.draw_couplings(n, 4) * 8
    grad, _ = _gpu_grad(tc, n, g, 1.05, 1.0, dt, steps, 5, atom=2)
    assert abs(grad[n] + grad[n + 1]) <= 1e-10 * max(abs(grad[n]), 1e-12)
    assert abs(grad[n]) > 1e-6
    gres, _ = _gpu_grad(tc, n, g, 1.0, 1.0, dt, steps, 5, atom=2)
    assert abs(gres[n]) < 1e-11 and abs(gres[n + 1]) < 1e-11


def test_qubit_photon_coupling_gradient(tc, oracle):
    n, steps, dt = 4, 10, 0.3
    g = W.draw_couplings(n, 6) * 8
    grad, _ = _gpu_grad(tc, n, g, 1.01, 1.0, dt, steps, 3, atom=2, coupling=1)
    ref = oracle.grad_forward(n, g, 1.01, 1.0, dt, steps, W.all_excited_state(n),
                              oracle.atom_population_operator(n, 2), coupling=oracle.COUPLING_QUBIT_PHOTON)
    assert np.max(np.abs(grad - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_autograd_function(tc):
    n, steps, dt = 4, 8, 0.3
    g = torch.tensor(W.draw_couplings(n, 1) * 8, dtype=torch.float64, requires_grad=True)
    wa = torch.tensor(1.02, dtype=torch.float64, requires_grad=True)
    wc = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    rho0 = torch.from_numpy(W.all_excited_rho(n)).cuda()
    s = np.arange(1 << n)
    O = torch.from_numpy(((s >> (n - 1)) & 1).astype(np.float64)).cuda()
    L = tc.EvolveFn.apply(g, wa, wc, rho0, O, dt, steps, 3)
    L.backward()
    ref, loss = _gpu_grad(tc, n, g.detach().numpy(), 1.02, 1.0, dt, steps, 3, atom=1)
    assert abs(L.item() - loss) < 1e-14
    np.testing.assert_allclose(g.grad.numpy(), ref[:n], rtol=0, atol=1e-14)
    assert abs(wa.grad.item() - ref[n]) < 1e-14 and abs(wc.grad.item() - ref[n + 1]) < 1e-14


def test_autograd_forward_runs_no_reverse_pass(tc, monkeypatch):
    """The forward of EvolveFn is the evolution alone: without a gradient
    request (no_grad, or inputs that need none) the reverse pass is never
    called; backward calls it once."""
    n, steps, dt = 4, 6, 0.3
    g0 = W.draw_couplings(n, 2) * 8
    _, loss = _gpu_grad(tc, n, g0, 1.01, 1.0, dt, steps, 3, atom=2)   # reference value, before counting
    calls = []
    real = tc.evolve_backward

    def counting(*args, **kw):
        calls.append(1)
        return real(*args, **kw)

    monkeypatch.setattr(tc, "evolve_backward", counting)
    rho0 = torch.from_numpy(W.all_excited_rho(n)).cuda()
    O = torch.from_numpy(((np.arange(1 << n) >> (n - 2)) & 1).astype(np.float64)).cuda()
    g = torch.tensor(g0, dtype=torch.float64)
    L_plain = tc.EvolveFn.apply(g, torch.tensor(1.01, dtype=torch.float64), torch.tensor(1.0, dtype=torch.float64),
                                rho0, O, dt, steps, 3)
    with torch.no_grad():
        gq = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
        L_nograd = tc.EvolveFn.apply(gq, torch.tensor(1.01, dtype=torch.float64),
                                     torch.tensor(1.0, dtype=torch.float64), rho0, O, dt, steps, 3)
    assert calls == [] and not L_plain.requires_grad
    assert abs(L_plain.item() - loss) < 1e-14 and abs(L_nograd.item() - loss) < 1e-14
    gr = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
    L = tc.EvolveFn.apply(gr, torch.tensor(1.01, dtype=torch.float64), torch.tensor(1.0, dtype=torch.float64),
                          rho0, O, dt, steps, 3)
    assert calls == []
    L.backward()
    assert calls == [1] and gr.grad is not None


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_autograd_function_matches_oracle_tangent(tc, oracle, precision):
    """EvolveFn in both product forms (FP64 DMMA and FP64 emulated on the BF16
    tensor cores, which needs n >= 7) against the oracle's forward-mode tangent."""
    n, steps, dt = 7, 20, 0.2
    g0 = W.draw_couplings(n, 12) * 6
    g = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
    wa = torch.tensor(1.02, dtype=torch.float64, requires_grad=True)
    wc = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    rho0 = torch.from_numpy(W.all_excited_rho(n)).cuda()
    Od = oracle.atom_population_operator(n, 1)
    L = tc.EvolveFn.apply(g, wa, wc, rho0, torch.from_numpy(Od).cuda(), dt, steps, 5, 0, precision)
    L.backward()
    ref = oracle.grad_forward(n, g0, 1.02, 1.0, dt, steps, W.all_excited_state(n), Od)
    got = np.concatenate([g.grad.numpy(), [wa.grad.item(), wc.grad.item()]])
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    _, obs = oracle.propagate(n, g0, 1.02, 1.0, dt, steps, W.all_excited_state(n))
    assert abs(L.item() - obs[-1, 0]) < 1e-12


def test_gradient_workload_n11(tc, oracle):
    """n = 11, dim 2048, 400 steps, checkpoints every 20: loss = P_1(T)."""
    cfg = W.config_n11_grad()
    grad, loss = _gpu_grad(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, cfg.ckpt_every,
                           atom=cfg.loss_atom)
    n = cfg.n
    O = oracle.atom_population_operator(n, cfg.loss_atom)
    psi0 = W.all_excited_state(n)
    ref = oracle.grad_forward(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, psi0, O)
    assert np.max(np.abs(grad - ref)) <= 1e-7 * np.max(np.abs(ref))
    # central differences of the oracle forward, h = 1e-6, three components
    h = 1e-6

    def L(g_, wa_, wc_):
        p, _ = oracle.propagate(n, g_, wa_, wc_, cfg.dt, cfg.steps, psi0, observe=False)
        return float(np.real(np.vdot(p, O * p)))

    fd = {}
    gp, gm = cfg.g.copy(), cfg.g.copy()
    gp[0] += h
    gm[0] -= h
    fd[0] = (L(gp, cfg.omega_a, cfg.omega_c) - L(gm, cfg.omega_a, cfg.omega_c)) / (2 * h)
    gp, gm = cfg.g.copy(), cfg.g.copy()
    gp[5] += h
    gm[5] -= h
    fd[5] = (L(gp, cfg.omega_a, cfg.omega_c) - L(gm, cfg.omega_a, cfg.omega_c)) / (2 * h)
    fd[n] = (L(cfg.g, cfg.omega_a + h, cfg.omega_c) - L(cfg.g, cfg.omega_a - h, cfg.omega_c)) / (2 * h)
    scale = max(abs(v) for v in fd.values())
    for j, v in fd.items():
        assert abs(grad[j] - v) <= 1e-6 * max(abs(v), scale), (j, grad[j], v)


@pytest.mark.parametrize("n,steps,ckpt", [(7, 12, 5), (9, 10, 4)])
def test_emulated_fp64_products_match_oracle_tangent(tc, oracle, n, steps, ckpt):
    """The per-step products on the BF16 tensor cores (exact digit slices): the same 1e-9 bound
    against the oracle tangent as the DMMA products."""
    g = W.draw_couplings(n, 70 + n) * 8
    wa, wc, dt = 1.03, 1.0, 0.3
    grad, loss = _gpu_grad(tc, n, g, wa, wc, dt, steps, ckpt, atom=2, precision="ozaki")
    O = oracle.atom_population_operator(n, 2)
    ref = oracle.grad_forward(n, g, wa, wc, dt, steps, W.all_excited_state(n), O)
    assert np.max(np.abs(grad - ref)) <= 1e-9 * np.max(np.abs(ref))
    g64, l64 = _gpu_grad(tc, n, g, wa, wc, dt, steps, ckpt, atom=2)
    assert abs(loss - l64) < 1e-13


def test_emulated_fp64_gradient_workload_n11(tc, oracle):
    """The n = 11 gradient workload with the emulated products, against the oracle tangent."""
    cfg = W.config_n11_grad()
    grad, loss = _gpu_grad(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, cfg.ckpt_every,
                           atom=cfg.loss_atom, precision="ozaki")
    n = cfg.n
    O = oracle.atom_population_operator(n, cfg.loss_atom)
    ref = oracle.grad_forward(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, W.all_excited_state(n), O)
    assert np.max(np.abs(grad - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_emulated_backward_rejects_small_n(tc):
    with pytest.raises(tc.TCError):
        _gpu_grad(tc, 5, W.draw_couplings(5, 1), 1.0, 1.0, 0.1, 3, 2, atom=1, precision="ozaki")
