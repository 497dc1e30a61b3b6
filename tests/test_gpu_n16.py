"""n = 16, dim 65536: 64 GiB per complex128 matrix.  U (64 GiB) and the
split-BF16 workspace (208 GiB: the operand parts of U, rho and X and their
FP32 planes) fill HBM, so rho stays in page-locked host memory: the
host-buffer call reads its rows with the SMs into the FP32 planes and parts
and writes rho' back through the buffer's mapping, with no device copy of rho
(TC_OP_EVOLVE_HOST_PINNED).  Two steps against the oracle's pure-state
propagation: observables and sampled entries within 1e-5.  The run takes a
process of its own (a fresh CUDA context: the ~5 GB of HBM left beside U and
the workspace is less than a long test process's context may hold) and is
skipped where the device or the host lacks the memory."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06937_gb300 as tc, workloads as W, oracle


def host_available():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


cfg = W.config_n16()
n, N, steps = cfg.n, cfg.N, 2
mat = 16 * N * N
work = tc.workspace_size(n, tc.PRECISIONS["bf16x3"], tc._abi.TC_OP_EVOLVE_HOST_PINNED, steps)
expm = tc.workspace_size(n, 0, tc._abi.TC_OP_EXPM_MODEL)
free, _ = torch.cuda.mem_get_info()
if free < mat + max(work, expm) + (512 << 20):
    print(json.dumps({"skip": "n = 16 needs %%.1f GB of free device memory (%%.1f free)"
                      %% ((mat + max(work, expm)) / 1e9, free / 1e9)}))
    sys.exit(0)
if host_available() < mat + (16 << 30):
    print(json.dumps({"skip": "n = 16 needs %%.0f GB of available host memory" %% (mat / 1e9)}))
    sys.exit(0)
p = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
U = tc.expm_model(p, cfg.dt)
torch.cuda.synchronize()
torch.cuda.empty_cache()   # the expm workspace goes back before the step's is taken
rho = torch.empty((N, N), dtype=torch.complex128, pin_memory=True)
rho.zero_()
rho[-1, -1] = 1.0
obs = torch.empty((steps + 1, tc.obs_stride(n)), dtype=torch.float64, pin_memory=True)
start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
start.record()
tc.evolve_host(U, rho, n, steps, "bf16x3", renorm_every=cfg.renorm_every, params=p, obs_host=obs)
end.record()
torch.cuda.synchronize()
seconds = start.elapsed_time(end) * 1e-3
del U
torch.cuda.empty_cache()
oracle.build()
psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, steps, W.all_excited_state(n))
o = obs.numpy()
e_obs = float(np.max(np.abs(o[:, :2 * n + 3] - oobs[:, :2 * n + 3])))
rng = np.random.default_rng(16)
top = np.argsort(-np.abs(psi))[:48]
ii = np.concatenate([rng.integers(0, N, 20000), np.repeat(top, len(top))])
jj = np.concatenate([rng.integers(0, N, 20000), np.tile(top, len(top))])
got = rho[torch.from_numpy(ii), torch.from_numpy(jj)].numpy()
e_rho = float(np.max(np.abs(got - psi[ii] * psi[jj].conj())))
print(json.dumps({"seconds": seconds, "steps": steps, "e_obs": e_obs, "e_rho": e_rho}))
"""


@pytest.fixture(scope="module")
def tc():
    from paper_2403_06937_gb300 import build
    build.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    return tc


def test_n16_split_bf16_host_buffer_against_oracle(tc, oracle):
    torch.cuda.synchronize()
    torch.cuda.empty_cache()   # this process's cached blocks go back before the child takes HBM
    out = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], capture_output=True, text=True, check=True)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    if "skip" in res:
        pytest.skip(res["skip"])
    print("n=16, %d steps through host rho, bf16x3: %.2f s (%.2f s/step), observables %.2e, rho sampled %.2e"
          % (res["steps"], res["seconds"], res["seconds"] / res["steps"], res["e_obs"], res["e_rho"]))
    assert res["e_obs"] < 1e-5 and res["e_rho"] < 1e-5
