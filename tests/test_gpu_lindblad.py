"""Parity of the open-system CUDA path (Eq. 5 with photon leakage, packed
excitation blocks) with the dense CPU oracle, through the C ABI.

Tolerances (FP64 throughout): propagators 1e-13 max-abs (unitary blocks,
Horner sums of a few hundred correctly rounded operations per entry, as the
closed expm); the state after 20 split steps 1e-12 max-abs (each step adds
rounding of order N u to entries of size <= 1, far below that bound for
N <= 128); the observable rows within the bound that state error e implies
for sums over the D x D state (D e for diagonal sums, 2 D e for the purity,
||H||_F D e for the energy).
"""
import math

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


@pytest.fixture(scope="module")
def L(oracle):
    from oracle import lindblad
    return lindblad


def _params(tc, n, g, wa, wc, coupling=0):
    return tc.Params(n, list(map(float, g)), wa, wc, coupling)


def _oracle_index(L, lay, k):
    """Oracle indices of block k's positions: (s, p = k - popcount(s))."""
    ix = L.index(lay.n)
    return [ix[(s, k - bin(s).count("1"))] for s in lay.basis[:lay.dims[k]]]


def _pack(L, lay, rho_full):
    out = np.zeros(lay.total, dtype=np.complex128)
    for k in range(lay.n + 1):
        sel = _oracle_index(L, lay, k)
        out[lay.offsets[k]:lay.offsets[k + 1]] = rho_full[np.ix_(sel, sel)].reshape(-1)
    return out


def _unpack(L, lay, packed):
    n = lay.n
    D = len(L.basis(n))
    full = np.zeros((D, D), dtype=np.complex128)
    for k in range(n + 1):
        sel = _oracle_index(L, lay, k)
        d = lay.dims[k]
        full[np.ix_(sel, sel)] = packed[lay.offsets[k]:lay.offsets[k + 1]].reshape(d, d)
    return full


def _random_block_rho(L, n, seed):
    rng = np.random.default_rng(seed)
    k = L.excitation_number(n)
    D = len(k)
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    rho = A @ A.conj().T
    rho[k[:, None] != k[None, :]] = 0.0
    return rho / np.trace(rho).real


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("coupling", [0, 1])
def test_propagators_match_oracle(tc, L, n, coupling):
    g = W.draw_couplings(n, 20 + n) * 10
    dt = 0.1
    lay = tc.lindblad_layout(n)
    U = tc.lindblad_propagators(_params(tc, n, g, 1.002, 1.0, coupling), dt).cpu().numpy()
    ref = L.propagator(n, g, 1.002, 1.0, dt, coupling)
    got = _unpack(L, lay, U)
    assert np.max(np.abs(got - ref)) < 1e-13
    for blk in lay.blocks(torch.from_numpy(U)):
        b = blk.numpy()
        assert np.array_equal(b, b.T)


@pytest.mark.parametrize("n,kappa,start", [(1, 0.3, "excited"), (3, 0.3, "excited"), (3, 0.0, "mixed"),
                                           (5, 0.25, "mixed"), (7, 0.4, "excited")])
def test_evolve_matches_oracle(tc, L, n, kappa, start):
    g = W.draw_couplings(n, 30 + n) * 20
    dt, steps = 0.1, 20
    lay = tc.lindblad_layout(n)
    p = _params(tc, n, g, 1.002, 1.0)
    rho0 = L.all_excited(n) if start == "excited" else _random_block_rho(L, n, 40 + n)
    U = tc.lindblad_propagators(p, dt)
    rho = torch.from_numpy(_pack(L, lay, rho0)).cuda()
    out, obs = tc.lindblad_evolve(p, kappa, dt, U, rho, steps)
    ref, rows = L.propagate(n, g, 1.002, 1.0, kappa, dt, steps, rho0)
    got = _unpack(L, lay, out.cpu().numpy())
    e = np.max(np.abs(got - ref))
    assert e < 1e-12
    # each observable is a sum over the D x D state: the diagonal sums move by
    # at most D e, the purity by 2 ||rho||_F ||d rho||_F <= 2 D e, the energy
    # by ||H||_F D e (Cauchy-Schwarz); e is the final, largest, state error
    D = got.shape[0]
    o = obs.cpu().numpy()
    bound = np.full(o.shape[1], D * e)
    bound[2 * n + 3] = 2 * D * e
    bound[2 * n + 4] = np.linalg.norm(L.hamiltonian(n, g, 1.002, 1.0)) * D * e
    assert np.all(np.abs(o - rows) <= bound + 1e-14)


def test_kappa_zero_top_block_is_the_closed_evolution(tc, L):
    """kappa = 0: block n evolves exactly as tc_evolve's FP64 path (reordered)."""
    n, dt, steps = 8, 0.1, 30
    g = W.draw_couplings(n, 50) * 5
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    N = 1 << n
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    top = lay.blocks(rho)[n]
    j = lay.basis.index(N - 1)
    top[j, j] = 1.0
    out, obs = tc.lindblad_evolve(p, 0.0, dt, tc.lindblad_propagators(p, dt), rho, steps)
    rho_c = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    rho_c[N - 1, N - 1] = 1.0
    Uc = tc.expm_model(p, dt)
    rc, obs_c = tc.evolve(Uc, rho_c, n, steps, "fp64", params=p)
    perm = torch.tensor(lay.basis, device="cuda")
    ref = rc[perm][:, perm]
    assert torch.max(torch.abs(lay.blocks(out)[n] - ref)).item() < 1e-12
    for k in range(n):
        assert torch.max(torch.abs(lay.blocks(out)[k])).item() == 0.0
    assert torch.max(torch.abs(obs[:, :-1] - obs_c[:, :-1])).item() < 1e-12
    assert torch.max(torch.abs(obs[:, -1] - obs_c[:, -1]) / torch.abs(obs_c[:, -1])).item() < 1e-11


def test_damped_jaynes_cummings_closed_form(tc, L):
    """n = 1 at resonance from |e, 0>: P_e(t) = e^{-kappa t / 2}(cos Wt + kappa/(4W) sin Wt)^2,
    W = sqrt(g^2 - kappa^2/16).  The split step converges to it at second
    order: halving dt divides the error over 0 <= t <= 7 by 4."""
    g, kappa, T = 0.3, 0.4, 7.0
    p = _params(tc, 1, [g], 1.0, 1.0)
    lay = tc.lindblad_layout(1)
    om = math.sqrt(g * g - kappa * kappa / 16.0)
    errs = []
    for dt in (0.02, 0.01):
        steps = int(round(T / dt))
        rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
        top = lay.blocks(rho)[1]
        j = lay.basis.index(1)
        top[j, j] = 1.0
        _, obs = tc.lindblad_evolve(p, kappa, dt, tc.lindblad_propagators(p, dt), rho, steps)
        t = np.arange(steps + 1) * dt
        ref = np.exp(-kappa * t / 2) * (np.cos(om * t) + kappa / (4 * om) * np.sin(om * t)) ** 2
        errs.append(np.max(np.abs(obs.cpu().numpy()[:, 0] - ref)))
    assert errs[1] < 2e-6
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


def test_invariants_n10(tc):
    """n = 10 (blocks up to 1024): trace 1, Hermitian blocks, populations in [0, 1],
    the mean excitation number falls and energy leaks with it."""
    n, dt, steps, kappa = 10, 0.05, 40, 0.5
    g = W.draw_couplings(n, 60) * 20
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    top = lay.blocks(rho)[n]
    j = lay.basis.index((1 << n) - 1)
    top[j, j] = 1.0
    out, obs = tc.lindblad_evolve(p, kappa, dt, tc.lindblad_propagators(p, dt), rho, steps)
    o = obs.cpu().numpy()
    assert np.max(np.abs(o[:, 2 * n + 2] - 1.0)) < 1e-12
    pm = o[:, n + 1:2 * n + 2]
    assert pm.min() > -1e-14
    assert np.max(np.abs(pm.sum(axis=1) - 1.0)) < 1e-12
    exc = o[:, :n].sum(axis=1) + o[:, n]   # sum P_i + <p> = <k>
    assert np.all(np.diff(exc) < 1e-14)
    assert exc[-1] < exc[0] - 0.05
    for blk in lay.blocks(out):
        assert torch.max(torch.abs(blk - blk.conj().T)).item() == 0.0


# ---------------------------------------------------------------- tensor-core forms
ACC = {"bf16x3": (6, 16), "tf32x3": (3, 8), "tf32": (1, 8)}   # part products, K per MMA


def lowp_step_bound(precision, K, vnorm, scale, n_damped):
    """One split step of a tensor-core form: the closed-form bound of the
    increment-form products, 2^-24 (4 + 2 n_acc 2 ||V||) max|rho| (TF32
    adding 4 2^-11 ||V|| max|rho| for its one-part operands), plus, for each
    of the two damping passes in FP32, (n + 1) rounded multiply-adds and one
    store per entry: 2 (n + 2) 2^-24 max|rho| (the channel's weights of one
    output sum to at most 1 / eta ~ 1, by Cauchy-Schwarz and the negative
    binomial series)."""
    prod, kstep = ACC[precision]
    n_acc = prod * K / kstep
    stores = 4.0 + (2.0 * (n_damped + 2) if n_damped else 0.0)
    b = 2.0 ** -24 * (stores + 2.0 * n_acc * 2.0 * vnorm) * scale
    if precision == "tf32":
        b += 4.0 * 2.0 ** -11 * vnorm * scale
    return b


def _block_vnorm(U):
    tr = np.trace(U)
    c = tr / abs(tr)
    return float(np.abs(U / c - np.eye(U.shape[0])).sum(1).max())


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_lowp_matches_oracle_n6(tc, L, precision):
    """n = 6 (blocks 1..64, each one padded tile), kappa = 0.3, 30 steps."""
    n, dt, steps, kappa = 6, 0.1, 30, 0.3
    g = W.draw_couplings(n, 70) * 20
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    rho0 = _random_block_rho(L, n, 71)
    Uo = L.propagator(n, g, 1.002, 1.0, dt)
    vnorm = max(_block_vnorm(Uo[np.ix_(sel, sel)]) for sel in (_oracle_index(L, lay, k) for k in range(n + 1)))
    U = tc.lindblad_propagators(p, dt)
    rho = torch.from_numpy(_pack(L, lay, rho0)).cuda()
    out, obs = tc.lindblad_evolve(p, kappa, dt, U, rho, steps, precision)
    ref, rows = L.propagate(n, g, 1.002, 1.0, kappa, dt, steps, rho0)
    got = _unpack(L, lay, out.cpu().numpy())
    scale = np.max(np.abs(rho0))
    tol = steps * lowp_step_bound(precision, 128, vnorm, scale, n)
    err = np.max(np.abs(got - ref))
    assert err < tol, (err, tol)
    D = got.shape[0]
    o = obs.cpu().numpy()
    assert np.max(np.abs(o[:, :n + 1] - rows[:, :n + 1])) < D * tol


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_lowp_matches_fp64_path_n8(tc, L, precision):
    """n = 8: blocks up to 256 (two tiles, ragged 163 / 219 / 247 / 255), against the
    FP64 open-system path (itself at oracle parity); ||V_k|| of the oracle's
    block propagators bounds the error."""
    n, dt, steps, kappa = 8, 0.05, 40, 0.4
    g = W.draw_couplings(n, 80) * 20
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    U = tc.lindblad_propagators(p, dt)
    vnorm = max(_block_vnorm(L.block_propagator(n, g, 1.002, 1.0, dt, k)[0]) for k in range(n + 1))
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    top = lay.blocks(rho)[n]
    j = lay.basis.index((1 << n) - 1)
    top[j, j] = 1.0
    ref, obs_ref = tc.lindblad_evolve(p, kappa, dt, U, rho, steps, "fp64")
    out, obs = tc.lindblad_evolve(p, kappa, dt, U, rho, steps, precision)
    tol = steps * lowp_step_bound(precision, 256, vnorm, 1.0, n)
    err = torch.max(torch.abs(out - ref)).item()
    assert err < tol, (err, tol)
    pops = torch.max(torch.abs(obs[:, :n] - obs_ref[:, :n])).item()
    assert pops < 1e-5   # the stated target of the split forms on populations


def test_lowp_renormalisation_n10(tc):
    """Split-BF16 at n = 10 with renormalisation every 10 steps: the total trace is
    back to 1 to FP32 rounding after each renormalisation, and the blocks stay Hermitian."""
    n, dt, steps, kappa = 10, 0.05, 30, 0.5
    g = W.draw_couplings(n, 90) * 20
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    top = lay.blocks(rho)[n]
    j = lay.basis.index((1 << n) - 1)
    top[j, j] = 1.0
    out, obs = tc.lindblad_evolve(p, kappa, dt, tc.lindblad_propagators(p, dt), rho, steps, "bf16x3",
                                  renorm_every=10)
    o = obs.cpu().numpy()
    for k in (10, 20, 30):
        assert abs(o[k, 2 * n + 2] - 1.0) < 1024 * 2.0 ** -24
    for blk in lay.blocks(out):
        assert torch.max(torch.abs(blk - blk.conj().T)).item() == 0.0
    exc = o[:, :n].sum(axis=1) + o[:, n]
    assert exc[-1] < exc[0] - 0.05


def test_errors(tc):
    import ctypes
    from paper_2403_06937_gb300 import _abi
    n = 4
    p = _params(tc, n, [0.1] * 4, 1.0, 1.0).c()
    lay = tc.lindblad_layout(n)
    U = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    rho = torch.zeros_like(U)
    w = torch.empty(1024, dtype=torch.uint8, device="cuda")
    lib = _abi.load()
    st = lib.tc_lindblad_evolve(ctypes.byref(p), 0.1, 0.1, ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(rho.data_ptr()), 3, 0, 0, None, ctypes.c_void_p(w.data_ptr()), 1024,
                                None)
    assert st == 3 and "need" in _abi.last_error()
    st = lib.tc_lindblad_evolve(ctypes.byref(p), -1.0, 0.1, ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(rho.data_ptr()), 3, 0, 0, None, ctypes.c_void_p(w.data_ptr()), 1024,
                                None)
    assert st == 1


# ---------------------------------------------------------------- FP64 emulated on the BF16 tensor cores
def test_emulated_fp64_matches_oracle_n6(tc, L):
    """Block products from exact digit slices: the FP64 form's 1e-12 against the oracle (each
    product is within K 2^-48 max|U| max|rho|, K = 128 here, far below that)."""
    n, dt, steps, kappa = 6, 0.1, 20, 0.3
    g = W.draw_couplings(n, 72) * 20
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    rho0 = _random_block_rho(L, n, 73)
    U = tc.lindblad_propagators(p, dt)
    rho = torch.from_numpy(_pack(L, lay, rho0)).cuda()
    out, obs = tc.lindblad_evolve(p, kappa, dt, U, rho, steps, "ozaki")
    ref, rows = L.propagate(n, g, 1.002, 1.0, kappa, dt, steps, rho0)
    got = _unpack(L, lay, out.cpu().numpy())
    assert np.max(np.abs(got - ref)) < 1e-12
    assert np.max(np.abs(obs.cpu().numpy()[:, :2 * n + 3] - rows[:, :2 * n + 3])) < 1e-11


def test_emulated_fp64_matches_fp64_path_n9(tc):
    """n = 9: blocks up to 512 (four tiles, ragged 382 / 466 / 502 / 511) against the DMMA blocks."""
    n, dt, steps, kappa = 9, 0.05, 10, 0.4
    g = W.draw_couplings(n, 74) * 20
    p = _params(tc, n, g, 1.002, 1.0)
    lay = tc.lindblad_layout(n)
    U = tc.lindblad_propagators(p, dt)
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    j = lay.basis.index((1 << n) - 1)
    lay.blocks(rho)[n][j, j] = 1.0
    a, oa = tc.lindblad_evolve(p, kappa, dt, U, rho, steps, "fp64")
    b, ob = tc.lindblad_evolve(p, kappa, dt, U, rho, steps, "ozaki")
    assert torch.max(torch.abs(a - b)).item() < 1e-12
    assert torch.max(torch.abs(oa - ob)[:, :2 * n + 3]).item() < 1e-11
    for blk in lay.blocks(b):
        assert torch.max(torch.abs(blk - blk.conj().T)).item() == 0.0
