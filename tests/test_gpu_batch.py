"""tc_batch_evolve: many systems of uneven size in one persistent launch per
product, the step loop captured in a CUDA graph.

Every system of a batch must give bitwise the result of tc_evolve on that
system alone: the batch kernel computes each 128 x 128 tile with the same
operand parts, the same order of part products and K slices, and the same
epilogue as the single-system kernel; FP64 runs the same DMMA products.
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


def _systems(tc, ns, seed, dt=0.05):
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(ns):
        g = rng.uniform(0.005, 0.015, size=n) * 6
        p = tc.Params(n, list(map(float, g)), 1.002, 1.0)
        U = tc.expm(tc.build_hamiltonian(p), n, dt)
        rho, _, _ = W.random_mixed_state(n, min(3, 1 << n), 100 + k)
        out.append((p, U, torch.from_numpy(rho).cuda()))
    return out


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32", "fp64", "ozaki"])
def test_batch_equals_standalone_runs(tc, precision):
    ns = [3, 9, 6, 7, 8, 9, 5, 7]
    sy = _systems(tc, ns, 1)
    steps = 4
    rhos, obs = tc.batch_evolve([s[1] for s in sy], [s[2] for s in sy], steps, precision,
                                params=[s[0] for s in sy])
    tc.sync_status()
    for (p, U, r0), rb, ob in zip(sy, rhos, obs):
        ra, oa = tc.evolve(U, r0, p.n, steps, precision, params=p)
        assert torch.equal(ra, rb), (p.n, (ra - rb).abs().max().item())
        assert torch.equal(oa, ob)


def test_batch_renormalisation_and_single_step(tc):
    ns = [7, 8]
    sy = _systems(tc, ns, 2)
    for steps in (1, 5):
        rhos, obs = tc.batch_evolve([s[1] for s in sy], [s[2] * 1.5 for s in sy], steps, "bf16x3",
                                    renorm_every=2, params=[s[0] for s in sy])
        for (p, U, r0), rb, ob in zip(sy, rhos, obs):
            ra, oa = tc.evolve(U, r0 * 1.5, p.n, steps, "bf16x3", renorm_every=2, params=p)
            assert torch.equal(ra, rb) and torch.equal(oa, ob)


def test_batch_of_64_workload_sample(tc):
    """64 systems, n ~ U{6..12} (seed 2), 200 steps, split-BF16: a sample of
    systems (the largest, the smallest and four more) against standalone runs."""
    cfgs = W.config_batch(steps=200)
    Us, rhos, ps = [], [], []
    for c in cfgs:
        p = tc.Params(c.n, list(map(float, c.g)), c.omega_a, c.omega_c)
        Us.append(tc.expm(tc.build_hamiltonian(p), c.n, c.dt))
        rhos.append(torch.from_numpy(W.all_excited_rho(c.n)).cuda())
        ps.append(p)
    out, obs = tc.batch_evolve(Us, rhos, cfgs[0].steps, "bf16x3", params=ps)
    tc.sync_status()
    ns = np.array([c.n for c in cfgs])
    pick = sorted({int(np.argmax(ns)), int(np.argmin(ns)), 5, 17, 33, 63})
    for k in pick:
        ra, oa = tc.evolve(Us[k], rhos[k], cfgs[k].n, cfgs[k].steps, "bf16x3", params=ps[k])
        assert torch.equal(ra, out[k]) and torch.equal(oa, obs[k]), k
        o = obs[k].cpu().numpy()
        n = cfgs[k].n
        assert abs(o[-1, 2 * n + 2] - 1.0) < 1e-5          # trace kept by the split form
