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


def test_batch_of_64_workload_against_oracle(tc, oracle):
    """Every system of the 64-system workload (n ~ U{6..12}, seed 2, 200 steps,
    split-BF16) against the oracle's pure-state propagation of that system
    (Eq. 6 for each one): populations, <p> and P(m) of every step within the
    split form's stated 1e-5, and the final rho on its largest entries and a
    random sample."""
    cfgs = W.config_batch(steps=200)
    Us, rhos, ps = [], [], []
    for c in cfgs:
        p = tc.Params(c.n, list(map(float, c.g)), c.omega_a, c.omega_c)
        Us.append(tc.expm(tc.build_hamiltonian(p), c.n, c.dt))
        rhos.append(torch.from_numpy(W.all_excited_rho(c.n)).cuda())
        ps.append(p)
    out, obs = tc.batch_evolve(Us, rhos, cfgs[0].steps, "bf16x3", params=ps)
    tc.sync_status()
    rng = np.random.default_rng(9)
    worst = 0.0
    for k, c in enumerate(cfgs):
        n = c.n
        psi, oobs = oracle.propagate(n, c.g, c.omega_a, c.omega_c, c.dt, c.steps, W.all_excited_state(n))
        o = obs[k].cpu().numpy()
        e_obs = float(np.max(np.abs(o[:, :2 * n + 2] - oobs[:, :2 * n + 2])))
        top = np.argsort(-np.abs(psi))[:16]
        ii = np.concatenate([rng.integers(0, c.N, 2000), np.repeat(top, len(top))])
        jj = np.concatenate([rng.integers(0, c.N, 2000), np.tile(top, len(top))])
        got = out[k][torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
        e_rho = float(np.max(np.abs(got - psi[ii] * psi[jj].conj())))
        worst = max(worst, e_obs, e_rho)
        assert e_obs < 1e-5 and e_rho < 1e-5, (k, n, e_obs, e_rho)
    print("64-system batch, 200 steps, split-BF16: max error vs oracle %.2e" % worst)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_mixed_state_batch_against_oracle_dense_step(tc, oracle, precision):
    """A batch of mixed states (n = 3..9) in the FP64 forms against the oracle's
    dense two-product step (Eq. 6 with its own U by columns): 1e-10 on rho
    after 5 steps."""
    ns = [3, 9, 6, 7, 8, 5, 9, 4]
    steps, dt = 5, 0.05
    rng = np.random.default_rng(21)
    Us, rhos, ps, gs, r0s = [], [], [], [], []
    for k, n in enumerate(ns):
        g = rng.uniform(0.005, 0.015, size=n) * 6
        p = tc.Params(n, list(map(float, g)), 1.002, 1.0)
        Us.append(tc.expm(tc.build_hamiltonian(p), n, dt))
        rho, _, _ = W.random_mixed_state(n, min(3, 1 << n), 300 + k)
        rhos.append(torch.from_numpy(rho).cuda())
        ps.append(p)
        gs.append(g)
        r0s.append(rho)
    out, _ = tc.batch_evolve(Us, rhos, steps, precision, params=ps)
    tc.sync_status()
    for k, n in enumerate(ns):
        Uo = oracle.expm(n, gs[k], 1.002, 1.0, dt)
        ref = r0s[k]
        for _ in range(steps):
            ref = oracle.dense_step(Uo, ref)
        err = float(np.max(np.abs(out[k].cpu().numpy() - ref)))
        assert err < 1e-10, (n, err)
