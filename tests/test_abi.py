"""The C-ABI library loads, exports every symbol include/tc.h declares, and
validates arguments on the host.  No compute call is made here (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tc.h")


def _declared():
    txt = open(HEADER).read()
    return re.findall(r"TC_API\s+[\w\s\*]+?\b(tc_\w+)\s*\(", txt)


@pytest.fixture(scope="module")
def lib():
    from paper_2403_06937_gb300 import build as B
    path = B.build()
    from paper_2403_06937_gb300 import _abi
    return _abi.load(path)


def test_header_declares_the_path_calls():
    names = set(_declared())
    for n in ("tc_build_hamiltonian", "tc_expm", "tc_evolve", "tc_observables", "tc_evolve_backward",
              "tc_workspace_size", "tc_last_error", "tc_sync_status"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lib._name)
    for name in _declared():
        assert hasattr(raw, name), name


def test_binding_covers_every_symbol(lib):
    from paper_2403_06937_gb300 import _abi
    assert set(_declared()) <= set(_abi.SIGNATURES)


def test_version_and_workspace_sizes(lib):
    from paper_2403_06937_gb300 import _abi
    assert b"sm_103a" in lib.tc_version()
    assert lib.tc_workspace_size(0, 0, 2, 0, 0) == 0
    assert lib.tc_workspace_size(17, 0, 2, 0, 0) == 0
    N = 1 << 10
    ev = lib.tc_workspace_size(10, _abi.TC_FP64, _abi.TC_OP_EVOLVE, 0, 0)
    assert ev >= 6 * N * N * 8
    ex = lib.tc_workspace_size(10, _abi.TC_FP64, _abi.TC_OP_EXPM, 0, 0)
    assert ex >= 13 * N * N * 8
    both = lib.tc_workspace_size(10, _abi.TC_FP64, _abi.TC_OP_EXPM | _abi.TC_OP_EVOLVE, 0, 0)
    assert both == max(ev, ex)


def test_pinned_host_workspace_skips_the_device_copy_of_rho(lib):
    """TC_OP_EVOLVE_HOST_PINNED: in the pipelined split forms (N >= 2048, a
    step or more) the host-buffer call on page-locked memory keeps no device
    copy of rho (16 N^2 bytes less); elsewhere it sizes the staging as
    TC_OP_EVOLVE_HOST does.  At n = 16 that is what fits beside U in HBM."""
    from paper_2403_06937_gb300 import _abi
    host, pinned = _abi.TC_OP_EVOLVE_HOST, _abi.TC_OP_EVOLVE_HOST_PINNED
    for n in (11, 12, 14, 16):
        for prec in (_abi.TC_BF16X3, _abi.TC_TF32, _abi.TC_TF32X3):
            full = lib.tc_workspace_size(n, prec, host, 2, 0)
            lean = lib.tc_workspace_size(n, prec, pinned, 2, 0)
            assert full - lean >= 16 * (1 << n) ** 2 - 256, (n, prec)
            assert lean >= lib.tc_workspace_size(n, prec, _abi.TC_OP_EVOLVE, 0, 0)
    for n, prec, steps in ((10, _abi.TC_BF16X3, 2), (12, _abi.TC_FP64, 2), (12, _abi.TC_FP64_OZAKI, 2),
                           (12, _abi.TC_BF16X3, 0)):
        assert lib.tc_workspace_size(n, prec, pinned, steps, 0) == lib.tc_workspace_size(n, prec, host, steps, 0)
    # n = 16, split-BF16: U (64 GiB) and the lean workspace stay below the 298 GB of HBM (284,208 MiB)
    # less the context, where the full host-buffer workspace does not
    U16 = 16 * (1 << 16) ** 2
    assert U16 + lib.tc_workspace_size(16, _abi.TC_BF16X3, pinned, 2, 0) < 296e9
    assert U16 + lib.tc_workspace_size(16, _abi.TC_BF16X3, host, 2, 0) > 298e9


def test_invalid_arguments_are_rejected_before_any_launch(lib):
    from paper_2403_06937_gb300 import _abi
    p = _abi.make_params(0, [], 1.0, 1.0)
    assert lib.tc_build_hamiltonian(ctypes.byref(p), ctypes.c_void_p(256), None) == 1
    assert b"outside" in lib.tc_last_error()
    p = _abi.make_params(3, [0.1, float("nan"), 0.1], 1.0, 1.0)
    assert lib.tc_build_hamiltonian(ctypes.byref(p), ctypes.c_void_p(256), None) == 1
    p = _abi.make_params(3, [0.1, 0.1, 0.1], 1.0, 1.0)
    assert lib.tc_build_hamiltonian(ctypes.byref(p), None, None) == 1
    assert lib.tc_build_hamiltonian(ctypes.byref(p), ctypes.c_void_p(264), None) == 1  # misaligned
    assert b"aligned" in lib.tc_last_error()
    # expm: bad dt, short workspace
    assert lib.tc_expm(ctypes.c_void_p(256), 3, -1.0, None, ctypes.c_void_p(512), None, 0, None) == 1
    assert lib.tc_expm(ctypes.c_void_p(256), 3, 0.1, None, ctypes.c_void_p(512), None, 0, None) == 3
    # evolve: unknown precision, negative steps
    assert lib.tc_evolve(ctypes.c_void_p(256), ctypes.c_void_p(512), 3, 1, 9, 0, None, None, None, 0, None) == 1
    assert lib.tc_evolve(ctypes.c_void_p(256), ctypes.c_void_p(512), 3, -1, 0, 0, None, None, None, 0, None) == 1


def test_no_device_means_unsupported_not_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert lib.tc_device_check() == 2
