"""tc_observables_noalloc: the observable reduction with its scratch in a
fixed device array, for callers that cannot allocate device memory (their
memory belongs to another allocator, or they cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree).  It must give exactly the row that
tc_observables gives with a caller-provided work buffer.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes alone in a fresh
process too (the first call on the device does its own set-up).
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2403_06937_gb300 import build
    build.build()
    from paper_2403_06937_gb300 import _abi
    lib = _abi.load()
    assert lib.tc_device_check() == 0
    return lib


def _with_work(lib, rho, n, params):
    from paper_2403_06937_gb300 import _abi
    out = torch.empty(2 * n + 5, dtype=torch.float64, device="cuda")
    nb = lib.tc_workspace_size(n, 0, _abi.TC_OP_OBSERVABLES, 0, 0)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = lib.tc_observables(ctypes.c_void_p(rho.data_ptr()), n, ctypes.byref(params), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(work.data_ptr()), nb, None)
    assert st == 0, _abi.last_error()
    return out


def _no_alloc(lib, rho, n, params):
    from paper_2403_06937_gb300 import _abi
    out = torch.empty(2 * n + 5, dtype=torch.float64, device="cuda")
    st = lib.tc_observables_noalloc(ctypes.c_void_p(rho.data_ptr()), n, ctypes.byref(params),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert st == 0, _abi.last_error()
    return out


@pytest.mark.parametrize("n", [3, 9, 12])
def test_no_alloc_matches_workspace_version_on_consecutive_calls(lib, oracle, n):
    from paper_2403_06937_gb300 import _abi
    g = W.draw_couplings(n, 31)
    params = _abi.make_params(n, g, 1.003, 0.998)
    if n <= 9:
        rho_a, _, _ = W.random_mixed_state(n, 3, 1)
        rho_b, _, _ = W.random_mixed_state(n, 2, 2)
    else:
        N = 1 << n
        rho_a = np.zeros((N, N), complex)
        rho_a[N - 1, N - 1] = 0.75
        rho_a[0, 0] = 0.25
        rho_b = W.all_excited_rho(n)
    ta = torch.from_numpy(rho_a).cuda()
    tb = torch.from_numpy(rho_b).cuda()
    # two calls in a row on different inputs: the second must not see the first's partials
    a1 = _no_alloc(lib, ta, n, params)
    b1 = _no_alloc(lib, tb, n, params)
    torch.cuda.synchronize()
    a0 = _with_work(lib, ta, n, params)
    b0 = _with_work(lib, tb, n, params)
    torch.cuda.synchronize()
    # the same kernels and the same fixed reduction order: bitwise the same rows
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    np.testing.assert_array_equal(b1.cpu().numpy(), b0.cpu().numpy())
    if n <= 9:
        np.testing.assert_allclose(a1.cpu().numpy(), oracle.observables(n, g, 1.003, 0.998, rho_a), atol=1e-12)


def test_no_alloc_rejects_bad_arguments(lib):
    from paper_2403_06937_gb300 import _abi
    params = _abi.make_params(4, [0.1] * 4, 1.0, 1.0)
    out = torch.empty(13, dtype=torch.float64, device="cuda")
    assert lib.tc_observables_noalloc(None, 4, ctypes.byref(params), ctypes.c_void_p(out.data_ptr()), None) == 1
    assert lib.tc_observables_noalloc(ctypes.c_void_p(out.data_ptr()), 17, None,
                                      ctypes.c_void_p(out.data_ptr()), None) == 1
