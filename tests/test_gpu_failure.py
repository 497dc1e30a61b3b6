"""Failure detection without a GPU fault.

* Timeout: a host-side injection makes a tensor-core launch withhold its first
  operand stage, so its consumer's (bounded) wait runs out; the kernel
  records TC_ERR_TIMEOUT, drains and returns, and the context stays usable.
* Non-finite or vanishing trace: the FP64 renormalisation records
  TC_ERR_NUMERIC instead of dividing by zero.
* A non-finite gradient is reported as TC_ERR_NUMERIC by the call itself.
"""
import ctypes

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
    tc.sync_status()
    return tc


def _setup(tc, n):
    g = W.draw_couplings(n, 1) * 4
    p = tc.Params(n, list(g), 1.01, 1.0)
    U = tc.expm(tc.build_hamiltonian(p), n, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 2)
    return p, U, torch.from_numpy(rho0).cuda()


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("n", [7, 8])
def test_injected_timeout_is_reported_and_context_survives(tc, precision, n):
    """n = 7: one tile, a single CTA; n = 8: 2 x 2 tiles, CTA pairs on the
    2-SM MMA (both CTAs of each pair withhold their first stage, the even
    CTA's MMA thread gives up, the abort reaches the odd CTA)."""
    from paper_2403_06937_gb300 import _abi
    p, U, r0 = _setup(tc, n)
    _abi.call("tc_fault_inject", 1, 1, 0.05)          # next launch: first stage withheld, 50 ms waits
    tc.evolve(U, r0, n, 1, precision, params=p)
    with pytest.raises(tc.TCError) as e:
        tc.sync_status()
    assert e.value.status == 5                        # TC_ERR_TIMEOUT
    tc.sync_status()                                  # the status word was cleared
    # the context is still usable and correct
    ref, _ = tc.evolve(U, r0, n, 2, "fp64", params=p)
    out, _ = tc.evolve(U, r0, n, 2, precision, params=p)
    tc.sync_status()
    assert (out - ref).abs().max().item() < 1e-6


def test_injection_argument_checks(tc):
    from paper_2403_06937_gb300 import _abi
    lib = _abi.load()
    assert lib.tc_fault_inject(7, 1, 0.1) == 1
    assert lib.tc_fault_inject(1, 1, 0.0) == 1
    assert lib.tc_fault_inject(1, 1, 60.0) == 1
    assert lib.tc_fault_inject(1, 0, 0.1) == 0        # count 0: nothing injected


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_vanishing_trace_is_a_numeric_error(tc, precision):
    n = 6
    p, U, r0 = _setup(tc, n)
    zero = torch.zeros_like(r0)
    tc.evolve(U, zero, n, 2, precision, renorm_every=1, params=p)
    with pytest.raises(tc.TCError) as e:
        tc.sync_status()
    assert e.value.status == 6                        # TC_ERR_NUMERIC
    tc.sync_status()


def test_non_finite_gradient_is_a_numeric_error(tc):
    n = 4
    p, U, r0 = _setup(tc, n)
    bad = r0.clone()
    bad[0, 0] = float("nan")
    s = np.arange(1 << n)
    O = torch.from_numpy(((s >> (n - 1)) & 1).astype(np.float64)).cuda()
    with pytest.raises(tc.TCError) as e:
        tc.evolve_backward(p, 0.1, 3, bad, U, O, ckpt_every=2)
    assert e.value.status == 6
