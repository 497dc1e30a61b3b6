"""tc_evolve_host with the tensor-core forms overlaps its transfers with the
first and last products: rho comes in by row blocks on a copy stream, the
first product of step 1 runs by column blocks as their rows arrive, and the
second product of the last step runs bottom-up by row bands, the entries
each band makes final converted and written out while the rows above are
computed (2 or 4 row blocks in and 2 to 8 row bands out from n = 11; below
that, whole copies around the loop).  A
page-locked rho_host is read and written by the SMs through its device
mapping; a pageable one goes through the copy engine and the device
staging.  The blocks run the same tile computations as the whole launches,
so the result equals the device-resident call bit for bit in both cases:
rho and the observable rows, with a renormalisation before or at the last
step."""
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


@pytest.mark.parametrize("n,prec,steps,renorm,pinned", [
    (10, "bf16x3", 2, 0, True),      # N < 2048: whole copies
    (10, "bf16x3", 2, 0, False),
    (11, "bf16x3", 1, 0, True),      # 2 blocks (16 tiles a side, raster group 8)
    (12, "bf16x3", 1, 0, True),      # 4 blocks
    (12, "bf16x3", 1, 0, False),
    (12, "bf16x3", 3, 2, True),      # renormalised in the middle, last step by blocks
    (12, "tf32x3", 2, 2, True),      # renormalised at the last step: blocks only for the way out
    (12, "tf32x3", 2, 2, False),
    (12, "tf32", 3, 0, True),
    (13, "bf16x3", 2, 0, True),      # 4 blocks in, 8 bands out
    (13, "bf16x3", 1, 0, False),
    (9, "fp64", 2, 0, True),
    (9, "fp64", 2, 0, False),
])
def test_host_path_equals_device_path(tc, n, prec, steps, renorm, pinned):
    p = tc.Params(n, list(map(float, W.draw_couplings(n, 21) * 5)), 1.01, 1.0)
    U = tc.expm_model(p, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 2, 50 + n)
    r_dev, o_dev = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, steps, prec, renorm_every=renorm, params=p)
    r_host = torch.from_numpy(rho0.copy())
    o_host = torch.empty((steps + 1, tc.obs_stride(n)), dtype=torch.float64)
    if pinned:
        r_host, o_host = r_host.pin_memory(), o_host.pin_memory()
    tc.evolve_host(U, r_host, n, steps, prec, renorm_every=renorm, params=p, obs_host=o_host)
    tc.sync_status()
    assert torch.equal(r_host, r_dev.cpu())
    assert torch.equal(o_host, o_dev.cpu())
    assert not np.array_equal(r_host.numpy(), rho0)   # the state did move
    del r_dev, o_dev, U
    torch.cuda.empty_cache()
