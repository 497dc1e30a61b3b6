"""Parity of tc_expm_model (e^{-iHdt} with H applied as a stencil, Sec. III.A
Eqs. 6-7) with the CPU oracle and with the dense tc_expm.

Tolerances: 1e-13 max-abs against the oracle (the same as the dense expm: a
unitary with O(1) entries, a few hundred correctly rounded FP64 operations
per entry); 1e-12 when squarings are forced (each squaring doubles the
error); Eq. 10 (fixed degree 10, no shift, no squaring) 1e-14 against the
oracle's dense Taylor sum.
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


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
@pytest.mark.parametrize("coupling", [0, 1])
def test_matches_oracle(tc, oracle, n, coupling):
    g = W.draw_couplings(n, 11 + n) * 3
    U = tc.expm_model(_params(tc, n, g, 1.002, 1.0, coupling), 0.05).cpu().numpy()
    ref = oracle.expm(n, g, 1.002, 1.0, 0.05, coupling)
    assert np.max(np.abs(U - ref)) < 1e-13
    assert np.array_equal(U, U.T)
    N = 1 << n
    assert np.max(np.abs(U.conj().T @ U - np.eye(N))) < 1e-13


def test_matches_dense_expm_n12(tc):
    """n = 12 workload couplings: the structured and the dense expm agree."""
    cfg = W.config_n12()
    p = _params(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c)
    Ud = tc.expm(tc.build_hamiltonian(p), cfg.n, cfg.dt)
    Um = tc.expm_model(p, cfg.dt)
    assert torch.max(torch.abs(Um - Ud)).item() < 1e-13
    del Ud, Um
    torch.cuda.empty_cache()


def test_paper_mode_is_eq10(tc, oracle):
    n, dt = 5, 0.1
    g = np.full(n, 0.01)
    U = tc.expm_model(_params(tc, n, g, 1.0, 1.0), dt, taylor_degree=10, squarings=0, shift=False).cpu().numpy()
    L = oracle.taylor_fixed(oracle.build_h(n, g, 1.0, 1.0), dt, 10)
    assert np.max(np.abs(U - (L + L.T) / 2)) < 1e-14


@pytest.mark.parametrize("dt,degree,squarings", [(0.2, 6, 3), (0.2, 12, 0), (2.0, 0, -1)])
def test_large_argument(tc, oracle, dt, degree, squarings):
    """||B|| from 0.7 to 8: the automatic plan squares, forced plans are honoured.

    The reference is the spectral U = V e^{-i w dt} V^T from the oracle's
    Jacobi eigensolver: an unscaled Taylor sum (the oracle's expm) loses
    about u e^{||H dt||} to cancellation at dt = 2.
    """
    n = 6
    g = W.draw_couplings(n, 3) * 4
    U = tc.expm_model(_params(tc, n, g, 1.01, 1.0), dt, taylor_degree=degree, squarings=squarings).cpu().numpy()
    w, V = oracle.jacobi_eig(oracle.build_h(n, g, 1.01, 1.0))
    ref = (V * np.exp(-1j * w * dt)[None, :]) @ V.T
    assert np.max(np.abs(U - ref)) < 1e-12


def test_uncoupled_resonant_is_a_phase(tc):
    """g = 0 and omega_a = omega_c: H = n omega I, U = e^{-i n omega dt} I."""
    n, dt, w = 4, 0.3, 1.25
    U = tc.expm_model(_params(tc, n, np.zeros(n), w, w), dt).cpu().numpy()
    phase = np.exp(-1j * n * w * dt)
    assert np.max(np.abs(U - phase * np.eye(1 << n))) < 1e-15


def test_short_workspace_is_an_error(tc):
    import ctypes
    from paper_2403_06937_gb300 import _abi
    n = 6
    p = _params(tc, n, W.draw_couplings(n, 1), 1.0, 1.0).c()
    U = torch.empty((64, 64), dtype=torch.complex128, device="cuda")
    w = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st = _abi.load().tc_expm_model(ctypes.byref(p), 0.1, None, ctypes.c_void_p(U.data_ptr()),
                                   ctypes.c_void_p(w.data_ptr()), 1024, None)
    assert st == 3
    assert "need" in _abi.last_error()


def test_n15_rows_are_unitary(tc):
    """n = 15 (dim 32768, the paper's largest): a sample of rows of U U^dag is the
    identity to 1e-13, and U is symmetric on the sampled block."""
    cfg = W.config_n15()
    p = _params(tc, cfg.n, cfg.g, cfg.omega_a, cfg.omega_c)
    U = tc.expm_model(p, cfg.dt)
    rows = torch.arange(0, 1 << cfg.n, 4093, device="cuda")
    G = U[rows] @ U[rows].conj().T
    assert torch.max(torch.abs(G - torch.eye(len(rows), dtype=G.dtype, device="cuda"))).item() < 1e-13
    assert torch.equal(U[rows][:, rows], U[rows][:, rows].T)
    del U, G
    torch.cuda.empty_cache()
