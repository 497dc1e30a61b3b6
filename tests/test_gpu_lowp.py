"""Parity of the tensor-core (tcgen05) forms with the FP64 path and the oracle.

Tolerances, from the arithmetic of the increment form (Y = P^H + V P^H with
V = U / c - I, c the unit phase of Tr U):
* rho and X are stored in FP32 (round to nearest): 2^-24 relative per store,
  two stores per step.
* The tensor cores accumulate V P^H in FP32 with truncation: at most one ulp
  (2^-23 relative) of a running sum bounded by ||V||_inf max|P| per
  accumulation, and there are `products x K / k_step` accumulations per
  element (BF16x3: 6 x K/16, TF32x3: 3 x K/8, TF32: K/8).
* The operand parts represent V and P to 2^-24 (split forms) or 2^-11 (TF32)
  relative, per operand of each of the two products.
So one step is within
    2^-24 (4 + 2 n_acc 2 ||V||) max|rho|      (split forms)
    (4 x 2^-11 ||V|| + 2^-24 (4 + 2 n_acc 2 ||V||)) max|rho|   (TF32)
and the stated target for the split-BF16 form is 1e-5 on populations.
TF32 does not meet that target (it is reported, not pinned); TF32x3 is its
remedy.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

ACC = {"bf16x3": (6, 16), "tf32x3": (3, 8), "tf32": (1, 8)}   # part products, K per MMA


def step_bound(precision, K, vnorm, scale):
    prod, kstep = ACC[precision]
    n_acc = prod * K / kstep
    b = 2.0 ** -24 * (4.0 + 2.0 * n_acc * 2.0 * vnorm) * scale
    if precision == "tf32":
        b += 4.0 * 2.0 ** -11 * vnorm * scale
    return b


def v_norm(U):
    """||U / c - I||_inf with c the unit phase of Tr U (a tolerance input only)."""
    tr = np.trace(U)
    c = tr / abs(tr)
    return float(np.abs(U / c - np.eye(U.shape[0])).sum(1).max())


@pytest.fixture(scope="module")
def tc():
    from paper_2403_06937_gb300 import build
    build.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    return tc


def _setup(tc, n, seed=3, scale=4.0, dt=0.1, wa=1.01, wc=1.0):
    g = W.draw_couplings(n, seed) * scale
    p = tc.Params(n, list(map(float, g)), wa, wc)
    U = tc.expm(tc.build_hamiltonian(p), n, dt)
    return g, p, U


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
@pytest.mark.parametrize("n", [3, 5, 7, 8, 10])
def test_one_step_matches_fp64(tc, oracle, n, precision):
    """n < 7 runs zero-padded in one 128 x 128 tile; n = 8, 10 span 2 x 2 and 8 x 8 tiles."""
    g, p, U = _setup(tc, n)
    rho0, _, _ = W.random_mixed_state(n, min(4, 1 << n), 11 + n)
    r0 = torch.from_numpy(rho0).cuda()
    ref, robs = tc.evolve(U, r0, n, 1, "fp64", params=p)
    out, obs = tc.evolve(U, r0, n, 1, precision, params=p)
    tc.sync_status()
    N = 1 << n
    vn = v_norm(oracle.expm(n, g, 1.01, 1.0, 0.1))
    scale = float(np.abs(rho0).max())
    bound = step_bound(precision, max(N, 128), vn, scale)
    err = (out - ref).abs().max().item()
    assert err < bound, (err, bound)
    # populations, <p>, P(m), trace are sums of at most N diagonal entries with
    # weights <= n; purity is bounded through |rho| <= scale.
    d = np.abs(obs.cpu().numpy() - robs.cpu().numpy())[1]
    assert np.all(d[:2 * n + 3] <= n * N * bound)
    assert d[2 * n + 3] <= 2 * N * N * scale * bound


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_result_is_exactly_hermitian(tc, precision):
    n = 9
    g, p, U = _setup(tc, n)
    rho0, _, _ = W.random_mixed_state(n, 3, 2)
    out, _ = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, 2, precision, params=p)
    o = out.cpu().numpy()
    assert np.array_equal(o, o.conj().T)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_n8_workload(tc, oracle, precision):
    """n = 8, 100 steps, from all-excited: populations against the oracle.

    Split forms: the stated target, 1e-5 on populations and on rho entries.
    TF32: within 100 times its one-step bound (reported, not the target).
    """
    cfg = W.config_n8()
    p = tc.Params(cfg.n, list(cfg.g), cfg.omega_a, cfg.omega_c)
    U = tc.expm(tc.build_hamiltonian(p), cfg.n, cfg.dt)
    rho0 = torch.from_numpy(W.all_excited_rho(cfg.n)).cuda()
    rho, obs = tc.evolve(U, rho0, cfg.n, cfg.steps, precision, params=p)
    tc.sync_status()
    psi, oobs = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps,
                                 W.all_excited_state(cfg.n))
    n = cfg.n
    o = obs.cpu().numpy()
    pop_err = np.max(np.abs(o[:, :2 * n + 2] - oobs[:, :2 * n + 2]))
    rho_err = np.max(np.abs(rho.cpu().numpy() - np.outer(psi, psi.conj())))
    if precision == "tf32":
        vn = v_norm(oracle.expm(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt))
        b = cfg.steps * step_bound(precision, cfg.N, vn, 1.0)
        assert rho_err < b and pop_err < n * b
    else:
        assert pop_err < 1e-5, pop_err
        assert rho_err < 1e-5, rho_err


def test_renormalisation_in_fp32_form(tc):
    n = 8
    g, p, U = _setup(tc, n)
    rho0, _, _ = W.random_mixed_state(n, 2, 5)
    rho, obs = tc.evolve(U, torch.from_numpy(1.5 * rho0).cuda(), n, 4, "bf16x3", renorm_every=2, params=p)
    o = obs.cpu().numpy()
    N = 1 << n
    assert abs(o[1, 2 * n + 2] - 1.5) < 1e-6      # one step: trace kept to FP32 level
    assert abs(o[2, 2 * n + 2] - 1.0) < N * 2.0 ** -24   # renormalised (FP32 storage of N entries)
    assert abs(o[4, 2 * n + 2] - 1.0) < N * 2.0 ** -24


def test_runs_are_bitwise_reproducible(tc):
    n = 9
    g, p, U = _setup(tc, n)
    rho0, _, _ = W.random_mixed_state(n, 3, 4)
    r0 = torch.from_numpy(rho0).cuda()
    a, oa = tc.evolve(U, r0, n, 3, "bf16x3", params=p)
    b, ob = tc.evolve(U, r0, n, 3, "bf16x3", params=p)
    assert torch.equal(a, b) and torch.equal(oa, ob)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_n12_against_fp64_path(tc, precision):
    cfg = W.config_n12()
    p = tc.Params(cfg.n, list(cfg.g), cfg.omega_a, cfg.omega_c)
    U = tc.expm(tc.build_hamiltonian(p), cfg.n, cfg.dt)
    rho0 = torch.from_numpy(W.all_excited_rho(cfg.n)).cuda()
    steps = 3
    ref, robs = tc.evolve(U, rho0, cfg.n, steps, "fp64", params=p)
    out, obs = tc.evolve(U, rho0, cfg.n, steps, precision, params=p)
    tc.sync_status()
    vn = 0.05       # ||V||_inf <= e^{||(H - mu) dt||} - 1 < 0.05 for this workload (dt = 0.05)
    tol = steps * step_bound(precision, cfg.N, vn, 1.0)       # max|rho0| = 1
    assert (out - ref).abs().max().item() < tol
    assert np.max(np.abs(obs.cpu().numpy() - robs.cpu().numpy())[:, :2 * cfg.n + 3]) < tol


def test_n14_workload_sampled_bf16x3(tc, oracle):
    """n = 14, dim 16384: the benchmark's launch configuration, a few steps, sampled entries."""
    cfg = W.config_n14()
    steps = 3
    p = tc.Params(cfg.n, list(cfg.g), cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)   # as the benchmark builds it
    rho0 = torch.zeros((cfg.N, cfg.N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    rho, obs = tc.evolve(U, rho0, cfg.n, steps, "bf16x3", renorm_every=cfg.renorm_every, params=p)
    tc.sync_status()
    psi, oobs = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, steps,
                                 W.all_excited_state(cfg.n))
    n = cfg.n
    o = obs.cpu().numpy()
    assert np.max(np.abs(o[:, :2 * n + 3] - oobs[:, :2 * n + 3])) < 1e-5
    rng = np.random.default_rng(5)
    idx = rng.integers(0, cfg.N, size=(20000, 2))
    top = np.argsort(-np.abs(psi))[:48]
    ii = torch.from_numpy(np.concatenate([idx[:, 0], np.repeat(top, len(top))])).cuda()
    jj = torch.from_numpy(np.concatenate([idx[:, 1], np.tile(top, len(top))])).cuda()
    got = rho[ii, jj].cpu().numpy()
    ii, jj = ii.cpu().numpy(), jj.cpu().numpy()
    want = psi[ii] * psi[jj].conj()
    assert np.max(np.abs(got - want)) < 1e-5


def _jc_excited(t, g, delta):
    """One atom of the qubit-photon reading from |e, 0>: the Rabi formula."""
    om2 = 4 * g * g + delta * delta
    return 1.0 - (4 * g * g / om2) * np.sin(np.sqrt(om2) * t / 2.0) ** 2


@pytest.mark.parametrize("n,precision,steps,tol", [(10, "fp64", 100, 1e-10), (14, "bf16x3", 100, 1e-5)])
def test_qubit_photon_closed_form(tc, n, precision, steps, tol):
    """Qubit-photon coupling: H = const + sum_i (Delta l_i + g_i sigma^x_i) factorises, so from the
    all-excited state every P_i(t) is the Rabi formula with its own g_i and P(m) is the
    Poisson-binomial distribution of the 1 - P_i.  An analytic pin of the whole dense path
    (H, U, the step loop, the observables) at the benchmark's size."""
    g = W.draw_couplings(n, 3) * 20
    wa, wc, dt = 1.002, 1.0, 0.05
    p = tc.Params(n, list(map(float, g)), wa, wc, 1)
    U = tc.expm_model(p, dt)
    N = 1 << n
    rho0 = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    _, obs = tc.evolve(U, rho0, n, steps, precision, renorm_every=50 if precision != "fp64" else 0, params=p)
    o = obs.cpu().numpy()
    t = np.arange(steps + 1) * dt
    P = np.stack([_jc_excited(t, gi, wa - wc) for gi in g], axis=1)
    assert np.max(np.abs(o[:, :n] - P)) < tol
    # P(m): the probability of m photons = m atoms relaxed, Poisson-binomial
    for r in (steps // 2, steps):
        dist = np.array([1.0])
        for q in 1.0 - P[r]:
            dist = np.convolve(dist, [1.0 - q, q])
        assert np.max(np.abs(o[r, n + 1:2 * n + 2] - dist)) < tol


def test_zero_steps_round_trip_is_one_fp32_rounding(tc):
    """The split forms store rho in FP32 planes: in and out again is one rounding, 2^-24 relative."""
    n = 6
    p = tc.Params(n, list(map(float, W.draw_couplings(n, 2))), 1.0, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 3, 4)
    r0 = torch.from_numpy(rho0).cuda()
    for precision in ("bf16x3", "tf32x3", "tf32"):
        rho, _ = tc.evolve(U, r0, n, 0, precision, params=p)
        d = (rho - r0).cpu().numpy()
        a = np.abs(rho0)
        assert np.all(np.abs(d.real) <= 2.0 ** -24 * np.abs(rho0.real))
        assert np.all(np.abs(d.imag) <= 2.0 ** -24 * np.abs(rho0.imag))
        assert a.max() > 0


# Max-abs error over all 500 steps of the n = 14 workload against the oracle:
# the split forms must meet the stated 1e-5 target; single-part TF32 is
# reported (its operands carry 11 bits) and held to a loose bound only.
N14_TARGET = {"bf16x3": 1e-5, "tf32x3": 1e-5, "tf32": 1e-3}


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_n14_500_steps_against_oracle(tc, oracle, precision):
    """The n = 14 workload over all 500 steps (renormalised every 50) against the
    oracle's pure-state propagation: populations, <p> and P(m) of every step,
    and the final rho on a random sample and the heaviest entries."""
    cfg = W.config_n14()
    n = cfg.n
    p = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    rho0 = torch.zeros((cfg.N, cfg.N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    rho, obs = tc.evolve(U, rho0, n, cfg.steps, precision, renorm_every=cfg.renorm_every, params=p)
    tc.sync_status()
    psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, W.all_excited_state(n))
    o = obs.cpu().numpy()
    e_pop = float(np.max(np.abs(o[:, :n] - oobs[:, :n])))
    e_obs = float(np.max(np.abs(o[:, :2 * n + 2] - oobs[:, :2 * n + 2])))
    rng = np.random.default_rng(14)
    top = np.argsort(-np.abs(psi))[:48]
    ii = np.concatenate([rng.integers(0, cfg.N, 20000), np.repeat(top, len(top))])
    jj = np.concatenate([rng.integers(0, cfg.N, 20000), np.tile(top, len(top))])
    got = rho[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    e_rho = float(np.max(np.abs(got - psi[ii] * psi[jj].conj())))
    print("n=14, 500 steps, %s: populations %.2e, populations/<p>/P(m) %.2e, rho sampled %.2e"
          % (precision, e_pop, e_obs, e_rho))
    assert e_obs < N14_TARGET[precision] and e_rho < N14_TARGET[precision]


@pytest.mark.slow
def test_n15_split_bf16_against_oracle(tc, oracle):
    """n = 15, dim 32768 (the paper's largest dimension; the inner dimension
    K = 32768 is accumulated in FP32 on the tensor cores), split-BF16, a few
    steps against the oracle: observables and sampled entries within 1e-5."""
    cfg = W.config_n15()
    n, steps = cfg.n, 3
    p = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    rho0 = torch.zeros((cfg.N, cfg.N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    rho, obs = tc.evolve(U, rho0, n, steps, "bf16x3", renorm_every=cfg.renorm_every, params=p)
    tc.sync_status()
    del U
    psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, steps, W.all_excited_state(n))
    o = obs.cpu().numpy()
    e_obs = float(np.max(np.abs(o[:, :2 * n + 3] - oobs[:, :2 * n + 3])))
    rng = np.random.default_rng(15)
    top = np.argsort(-np.abs(psi))[:48]
    ii = np.concatenate([rng.integers(0, cfg.N, 20000), np.repeat(top, len(top))])
    jj = np.concatenate([rng.integers(0, cfg.N, 20000), np.tile(top, len(top))])
    got = rho[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    e_rho = float(np.max(np.abs(got - psi[ii] * psi[jj].conj())))
    print("n=15, %d steps, bf16x3: observables %.2e, rho sampled %.2e" % (steps, e_obs, e_rho))
    assert e_obs < 1e-5 and e_rho < 1e-5


def test_cta_pairs_give_the_same_bits_as_single_ctas(tc, tmp_path):
    """The 2-SM MMA arrangement (CTA pairs of two row tiles, each CTA loading
    its own U rows and half of every B part) against single CTAs
    (TC_GEMM_PAIRS=0), every split form: each tile's MMAs take the same
    operands in the same order, so every output bit is the same.  n = 8, 10,
    12 (2, 8 and 32 tiles a side), three steps, mixed states."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for mode in ("0", "1"):
        path = str(tmp_path / ("tc_pairs_%s.npz" % mode))
        script = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06937_gb300 as tc, workloads as W
res = {}
for prec in ('bf16x3', 'tf32x3', 'tf32'):
    for n in (8, 10, 12):
        p = tc.Params(n, list(map(float, W.draw_couplings(n, 11) * 5)), 1.01, 1.0)
        U = tc.expm_model(p, 0.1)
        rho0, _, _ = W.random_mixed_state(n, 2, 40 + n)
        r, o = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, 3, prec, params=p)
        tc.sync_status()
        res['rho_%%s_%%d' %% (prec, n)] = r.cpu().numpy()
        res['obs_%%s_%%d' %% (prec, n)] = o.cpu().numpy()
np.savez(%r, **res)
""" % (root, path)
        subprocess.run([sys.executable, "-c", script], env=dict(os.environ, TC_GEMM_PAIRS=mode), check=True)
        out[mode] = np.load(path)
    for key in out["0"].files:
        assert np.array_equal(out["0"][key], out["1"][key]), key
