"""Parity of the FP64-accurate tensor-core form (TC_FP64_OZAKI: exact integer
slices on the BF16 tensor cores) with the FP64 DMMA path and the oracle.

Tolerance, from the arithmetic: every entry x of an operand row with scale
2^e (max |x| < 2^(e-1)) is held to 2^(e-55) (one rounding of x 2^(54-e) to an
integer), the slice-pair sums are exact, and the dropped pairs (t + u >= 9)
contribute at most 8 * 2^10 * 2^-66 2^(e_i + f_j) per term; with
2^e <= 4 max|row| each of the K terms of a product is within
2^-48 max|A_i| max|B_j|, so one product is within K 2^-48 max|U| max|P|,
two products per step.  (The FP64 DMMA reference adds its own K 2^-53.)
That is the bound of the 6-bit digits (K > 4096); the 7- and 8-bit digits of
the smaller sizes (56 bits, dropped pairs below 2^-51.2 of the scales) meet
it with room to spare.  It is a worst case, loose enough that a dropped top
slice level would pass it: test_single_product_tight checks the typical size
of the error instead.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def bound(n, steps, umax=1.0, pmax=1.0):
    K = max(1 << n, 128)
    return steps * 2 * K * 2.0 ** -48 * umax * pmax * 1.01 + steps * 2 * K * 2.0 ** -53


@pytest.fixture(scope="module")
def tc():
    from paper_2403_06937_gb300 import build
    build.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    return tc


def _params(tc, n, g, wa, wc, coupling=0):
    return tc.Params(n, list(map(float, g)), wa, wc, coupling)


@pytest.mark.parametrize("n,steps", [(1, 30), (3, 20), (6, 20), (7, 10), (9, 10), (10, 5)])
def test_matches_fp64_path(tc, n, steps):
    g = W.draw_couplings(n, 60 + n) * 5
    p = _params(tc, n, g, 1.013, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, min(3, 1 << n), 30 + n)
    r0 = torch.from_numpy(rho0).cuda()
    a, oa = tc.evolve(U, r0, n, steps, "fp64", params=p)
    b, ob = tc.evolve(U, r0, n, steps, "ozaki", params=p)
    tc.sync_status()
    umax = torch.max(torch.abs(U)).item()
    tol = bound(n, steps, umax, 1.0)
    assert torch.max(torch.abs(a - b)).item() < tol
    assert torch.max(torch.abs(oa - ob)[:, :2 * n + 3]).item() < (1 << n) * tol
    assert torch.equal(b, b.conj().T)   # exactly Hermitian: the upper half is the mirrored lower half


def test_n8_workload_against_oracle(tc, oracle):
    """n = 8, 100 steps from the all-excited state: the FP64 target 1e-10 on rho and the rows."""
    cfg = W.config_n8()
    n = cfg.n
    p = _params(tc, n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    rho0 = torch.from_numpy(W.all_excited_rho(n)).cuda()
    rho, obs = tc.evolve(U, rho0, n, cfg.steps, "ozaki", params=p)
    psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, W.all_excited_state(n))
    assert np.max(np.abs(rho.cpu().numpy() - np.outer(psi, psi.conj()))) < 1e-10
    assert np.max(np.abs(obs.cpu().numpy() - oobs)) < 1e-10


def test_runs_are_bitwise_reproducible(tc):
    n = 8
    p = _params(tc, n, W.draw_couplings(n, 4) * 10, 1.0, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 9)
    r0 = torch.from_numpy(rho0).cuda()
    a, oa = tc.evolve(U, r0, n, 7, "ozaki", params=p)
    b, ob = tc.evolve(U, r0, n, 7, "ozaki", params=p)
    assert torch.equal(a, b) and torch.equal(oa, ob)


def test_zero_steps_and_tiny_rows(tc):
    """Zero steps return rho unchanged (FP64 storage); a state scaled by 2^-950 keeps its relative
    accuracy (its rows' 2^(54 - e) exceeds the FP64 exponent range and is applied as two factors;
    the smallest slice products, 2^(e_i + e_j - 60), stay normal)."""
    n = 5
    p = _params(tc, n, W.draw_couplings(n, 5), 1.0, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 3)
    r0 = torch.from_numpy(rho0).cuda()
    out, _ = tc.evolve(U, r0, n, 0, "ozaki", params=p)
    assert torch.equal(out, r0)
    tiny = r0 * 2.0 ** -950
    a, _ = tc.evolve(U, tiny, n, 2, "fp64", params=p)
    b, _ = tc.evolve(U, tiny, n, 2, "ozaki", params=p)
    assert torch.max(torch.abs(a - b)).item() < 2.0 ** -950 * bound(n, 2, 1.0, 1.0)
    assert torch.max(torch.abs(b)).item() > 2.0 ** -960


def test_n12_workload_against_fp64_path(tc):
    cfg = W.config_n12()
    n = cfg.n
    p = _params(tc, n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    N = 1 << n
    rho0 = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    a, oa = tc.evolve(U, rho0, n, 3, "fp64", params=p)
    b, ob = tc.evolve(U, rho0, n, 3, "ozaki", params=p)
    assert torch.max(torch.abs(a - b)).item() < bound(n, 3)
    assert torch.max(torch.abs(oa - ob)).item() < bound(n, 3) * 64


def test_n14_workload_sampled(tc, oracle):
    """n = 14 (the benchmark's size), 3 steps: sampled entries and the observable rows against the
    oracle's pure-state propagation."""
    cfg = W.config_n14()
    n = cfg.n
    p = _params(tc, n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    rho0 = torch.zeros((cfg.N, cfg.N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    steps = 3
    rho, obs = tc.evolve(U, rho0, n, steps, "ozaki", params=p)
    tc.sync_status()
    psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, steps, W.all_excited_state(n))
    tol = bound(n, steps) + 1e-13
    assert np.max(np.abs(obs.cpu().numpy()[:, :2 * n + 3] - oobs[:, :2 * n + 3])) < tol
    rng = np.random.default_rng(7)
    idx = rng.integers(0, cfg.N, size=(20000, 2))
    top = np.argsort(-np.abs(psi))[:48]
    ii = np.concatenate([idx[:, 0], np.repeat(top, len(top))])
    jj = np.concatenate([idx[:, 1], np.tile(top, len(top))])
    got = rho[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    assert np.max(np.abs(got - psi[ii] * psi[jj].conj())) < tol
    del rho, rho0, U
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_n15_one_step_two_k_chunks(tc, oracle):
    """n = 15: K = 32768 is summed in two exact passes of 16384 per slice pair."""
    cfg = W.config_n15()
    n = cfg.n
    p = _params(tc, n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    rho0 = torch.zeros((cfg.N, cfg.N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    rho, obs = tc.evolve(U, rho0, n, 1, "ozaki", params=p)
    tc.sync_status()
    psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, 1, W.all_excited_state(n))
    tol = bound(n, 1) + 1e-13
    assert np.max(np.abs(obs.cpu().numpy()[:, :2 * n + 3] - oobs[:, :2 * n + 3])) < tol
    top = np.argsort(-np.abs(psi))[:64]
    ii, jj = np.repeat(top, len(top)), np.tile(top, len(top))
    got = rho[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    assert np.max(np.abs(got - psi[ii] * psi[jj].conj())) < tol
    del rho, rho0, U
    torch.cuda.empty_cache()


def test_host_buffers_and_renormalisation(tc):
    """tc_evolve_host with the emulated form (rho in pinned host memory) equals the device call;
    renormalisation divides by the FP64 trace."""
    n = 7
    p = _params(tc, n, W.draw_couplings(n, 8) * 5, 1.01, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 12)
    r_dev, o_dev = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, 6, "ozaki", params=p)
    r_host = torch.from_numpy(rho0.copy()).pin_memory()
    o_host = torch.empty((7, 2 * n + 5), dtype=torch.float64).pin_memory()
    tc.evolve_host(U, r_host, n, 6, "ozaki", params=p, obs_host=o_host)
    assert torch.equal(r_host, r_dev.cpu())
    assert torch.equal(o_host, o_dev.cpu())
    half = torch.from_numpy(rho0 * 0.5).cuda()
    rr, oo = tc.evolve(U, half, n, 4, "ozaki", renorm_every=2, params=p)
    tr = oo[:, 2 * n + 2].cpu().numpy()
    assert abs(tr[0] - 0.5) < 1e-15 and np.max(np.abs(tr[2:] - 1.0)) < 1e-14


def _uuh(tc, n, precision, seed=3):
    """One step from rho0 = I is the single product U U^H (the first product,
    U I, only rounds U to its slice grid): U a random complex symmetric matrix
    (the form every e^{-iH dt} of a real symmetric H has, which the FP64 path
    relies on), max |U| = 1."""
    N = 1 << n
    rng = np.random.default_rng(seed + n)
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    U = (A + A.T) / 2
    U /= np.max(np.abs(U))
    Ud = torch.from_numpy(U).cuda()
    p = _params(tc, n, W.draw_couplings(n, 2), 1.0, 1.0)
    eye = torch.eye(N, dtype=torch.complex128, device="cuda")
    out, _ = tc.evolve(Ud, eye, n, 1, precision, params=p)
    tc.sync_status()
    return U, out


def _tight(K, ref):
    """Off the diagonal 16 sqrt(K) 2^-53 of the operand scales (max |U| = 1)
    plus 16 units of 2^-53 |entry|; on it (a coherent sum of K positive
    terms, which an FP64 reference summing in sequence rounds K times at the
    size of the sum) 16 sqrt(K) 2^-53 |entry| in addition."""
    base = 16 * np.sqrt(K) * 2.0 ** -53
    tol = base + 16 * 2.0 ** -53 * np.abs(ref)
    i = np.arange(ref.shape[0])
    tol[i, i] += base * np.abs(ref[i, i])
    return tol


def _ratio(got, ref, K):
    return float(np.max(np.abs(got - ref) / _tight(K, ref)))


@pytest.mark.parametrize("n", [7, 10, 11, 12, 13])
def test_single_product_tight(tc, n):
    """U U^H against numpy (blocked FP64 sums; up to n = 12) within _tight.
    A CPU emulation of the exact slice arithmetic (test_ozaki_digit_scheme.py)
    puts a correct product at
    0.04-0.2 of that bound (7- and 8-bit digits at the low end, 6-bit at the
    high end) and numpy's at about 0.2; leaving out the top slice level
    (t + u = S - 1) would put it at 5-16 times the bound: this catches that
    where the worst-case bound above cannot.  Against the FP64 DMMA path,
    whose K-term sums run in sequence (an error near K 2^-53 of the operand
    scales, measured 0.27 K 2^-53 at n = 13), the bound adds K 2^-53."""
    K = max(1 << n, 128)
    U, oz = _uuh(tc, n, "ozaki")
    got = oz.cpu().numpy()
    if n <= 12:
        r = _ratio(got, U @ U.conj().T, K)
        print("n=%d: error / bound %.3f against numpy" % (n, r))
        assert r < 1.0
    _, ref = _uuh(tc, n, "fp64")
    ref = ref.cpu().numpy()
    d = np.max(np.abs(got - ref) / (_tight(K, ref) + K * 2.0 ** -53))
    print("n=%d: error / bound %.3f against the FP64 path" % (n, d))
    assert d < 1.0
    assert torch.equal(oz, oz.conj().T)
    del oz
    torch.cuda.empty_cache()


def test_six_bit_digits_at_every_size(tc, tmp_path):
    """TC_OZ_BITS=6 keeps the 6-bit digits (9 slices, 45 pairs) at the sizes
    that default to 8- and 7-bit ones (n = 10, 12): the same tight bound
    against numpy holds, and the low bits differ from the default form's, so
    the setting took effect."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for n in (10, 12):
        path = str(tmp_path / ("six_%d.npy" % n))
        script = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
sys.path.insert(0, %r)
import paper_2403_06937_gb300 as tc
from test_gpu_ozaki import _uuh
_, out = _uuh(tc, %d, 'ozaki')
np.save(%r, out.cpu().numpy())
""" % (root, os.path.join(root, "tests"), n, path)
        subprocess.run([sys.executable, "-c", script], env=dict(os.environ, TC_OZ_BITS="6"), check=True)
        six = np.load(path)
        U, wide = _uuh(tc, n, "ozaki")
        wide = wide.cpu().numpy()
        ref = U @ U.conj().T
        r6, rw = _ratio(six, ref, 1 << n), _ratio(wide, ref, 1 << n)
        print("n=%d: error / bound %.3f (6-bit digits), %.3f (default)" % (n, r6, rw))
        assert r6 < 1.0 and rw < 1.0
        assert not np.array_equal(six, wide)


def test_cta_pairs_give_the_same_bits_as_single_ctas(tc, tmp_path):
    """The 2-SM MMA arrangement (CTA pairs of two row tiles, each CTA loading
    its own U rows and half of the P panel) against single CTAs
    (TC_OZ_PAIRS=0): the integer slice sums are the same, so every output
    bit is.  n = 8, 10, 12 (2, 8 and 32 tiles a side), three steps each,
    mixed states, both products of the step."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for mode in ("0", "1"):
        path = str(tmp_path / ("pairs_%s.npz" % mode))
        script = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06937_gb300 as tc, workloads as W
res = {}
for n in (8, 10, 12):
    p = tc.Params(n, list(map(float, W.draw_couplings(n, 11) * 5)), 1.01, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 40 + n)
    r, o = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, 3, 'ozaki', params=p)
    tc.sync_status()
    res['rho%%d' %% n] = r.cpu().numpy()
    res['obs%%d' %% n] = o.cpu().numpy()
np.savez(%r, **res)
""" % (root, path)
        subprocess.run([sys.executable, "-c", script], env=dict(os.environ, TC_OZ_PAIRS=mode), check=True)
        out[mode] = np.load(path)
    for key in out["0"].files:
        assert np.array_equal(out["0"][key], out["1"][key]), key


def test_cta_pairs_with_odd_tile_counts_give_the_same_bits(tc, tmp_path):
    """The open system's excitation blocks at n = 9 have 1, 3 and 4 tiles a
    side; with an odd count the odd CTA of the last row pair has no rows (its
    U loads read zeros, it writes nothing).  Pairs against single CTAs
    (TC_OZ_PAIRS=0), three split steps with photon leakage: every bit equal."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for mode in ("0", "1"):
        path = str(tmp_path / ("odd_%s.npz" % mode))
        script = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06937_gb300 as tc, workloads as W
n = 9
p = tc.Params(n, list(map(float, W.draw_couplings(n, 13) * 5)), 1.002, 1.0)
U = tc.lindblad_propagators(p, 0.05)
lay = tc.lindblad_layout(n)
assert any((-(-d // 128)) %% 2 == 1 and d > 128 for d in lay.dims)
rho = torch.zeros(lay.total, dtype=torch.complex128, device='cuda')
rng = np.random.default_rng(17)
for blk in lay.blocks(rho):
    d = blk.shape[0]
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    M = A @ A.conj().T
    blk.copy_(torch.from_numpy(M / np.trace(M).real / (n + 1)))
r, o = tc.lindblad_evolve(p, 0.05, 0.05, U, rho, 3, 'ozaki')
tc.sync_status()
np.savez(%r, rho=r.cpu().numpy(), obs=o.cpu().numpy())
""" % (root, path)
        subprocess.run([sys.executable, "-c", script], env=dict(os.environ, TC_OZ_PAIRS=mode), check=True)
        out[mode] = np.load(path)
    for key in out["0"].files:
        assert np.array_equal(out["0"][key], out["1"][key]), key
