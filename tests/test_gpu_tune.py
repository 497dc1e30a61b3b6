"""tc_autotune: picks a built configuration; results do not depend on it."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tc():
    from paper_2403_06937_gb300 import build
    build.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    return tc


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32", "fp64"])
def test_tuning_changes_speed_not_results(tc, precision):
    n = 10 if precision != "fp64" else 9
    g = W.draw_couplings(n, 2) * 4
    p = tc.Params(n, list(g), 1.01, 1.0)
    U = tc.expm(tc.build_hamiltonian(p), n, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 3, 3)
    r0 = torch.from_numpy(rho0).cuda()
    before, ob = tc.evolve(U, r0, n, 3, precision, params=p)
    choice = tc.autotune(n, precision)
    assert choice == tc.autotune_lookup(n, precision)
    if precision == "fp64":
        assert choice["f64_tile"] in (32, 64)
    else:
        assert choice["tc_group"] in (4, 8, 12, 16)
        assert choice["tc_stages"] in {"bf16x3": (4, 3), "tf32x3": (6, 3), "tf32": (8, 4)}[precision]
        assert choice["tc_shape"] in (1, 2, 3)
    after, oa = tc.evolve(U, r0, n, 3, precision, params=p)
    assert torch.equal(before, after) and torch.equal(ob, oa)


def test_both_fp64_tiles_agree(tc, oracle, tmp_path):
    """The 32 and 64 DMMA tiles (forced through the cache) give the same step."""
    n = 8
    g = W.draw_couplings(n, 5) * 4
    rho0, wts, states = W.random_mixed_state(n, 2, 1)
    res = []
    for tile in (32, 64):
        path = str(tmp_path / ("tune_tile_%d.jsonl" % tile))
        arch = 103
        with open(path, "w") as f:
            f.write('{"arch": %d, "n": %d, "precision": 0, "f64_tile": %d, "tc_group": 8, "tc_stages": 0}\n'
                    % (arch, n, tile))
        script = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06937_gb300 as tc, workloads as W
n = %d
g = W.draw_couplings(n, 5) * 4
p = tc.Params(n, list(g), 1.01, 1.0)
assert tc.autotune_lookup(n, 'fp64')['f64_tile'] == %d
U = tc.expm(tc.build_hamiltonian(p), n, 0.1)
rho0, _, _ = W.random_mixed_state(n, 2, 1)
out, _ = tc.evolve(U, torch.from_numpy(rho0).cuda(), n, 3, 'fp64', params=p)
np.save(%r, out.cpu().numpy())
""" % (ROOT, n, tile, path + ".npy")
        env = dict(os.environ, TC_AUTOTUNE_CACHE=path)
        subprocess.run([sys.executable, "-c", script], env=env, check=True)
        res.append(np.load(path + ".npy"))
    finals = [oracle.propagate(n, g, 1.01, 1.0, 0.1, 3, s_, observe=False)[0] for s_ in states]
    ref = sum(w * np.outer(f, f.conj()) for w, f in zip(wts, finals))
    for r in res:
        assert np.max(np.abs(r - ref)) < 1e-12
    assert np.max(np.abs(res[0] - res[1])) < 1e-15
