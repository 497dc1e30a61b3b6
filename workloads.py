"""Seeded synthetic inputs for the Tavis-Cummings workloads.

This module holds no arithmetic of the method: it only draws the model
parameters and initial states, so that the CUDA library and the CPU oracle are
fed identical inputs.  Random couplings are drawn here with numpy's PCG64
generator and passed in; neither side draws random numbers itself.

The paper (arXiv 2403.06937) states no coupling, frequency, time step or step
count; the five workloads below fix them.  Their sizes are the paper's own
dimensions 2^8 .. 2^14 (Tables I-II).

Index convention used throughout: atom i (1-based) is bit (n - i) of the basis
index, so atom 1 is the most significant bit; the photon number of basis
state s is n - popcount(s).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class TCConfig:
    name: str
    n: int
    g: np.ndarray
    omega_a: float
    omega_c: float
    dt: float
    steps: int
    renorm_every: int = 0
    ckpt_every: int = 0
    loss_atom: int = 0
    description: str = ""
    kappa: float = 0.0     # photon leakage rate of the open-system form (0: closed)

    @property
    def N(self) -> int:
        return 1 << self.n


def draw_couplings(n: int, seed: int, lo: float = 0.005, hi: float = 0.015) -> np.ndarray:
    """g_i i.i.d. uniform [lo, hi), numpy default_rng(seed)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def config_n8() -> TCConfig:
    """n = 8 atoms, dim 256: equal g = 0.01, resonant, dt = 0.1, 100 steps."""
    return TCConfig("n8_fp64", 8, np.full(8, 0.01), 1.0, 1.0, 0.1, 100,
                    description="n=8, dim 256, g_i=0.01, w_a=w_c=1, dt=0.1, 100 steps")


def config_n12() -> TCConfig:
    """n = 12, dim 4096: g ~ U[0.005, 0.015] (seed 0), w_a - w_c = 0.002."""
    return TCConfig("n12_fp64", 12, draw_couplings(12, 0), 1.002, 1.0, 0.05, 200,
                    description="n=12, dim 4096, g~U[0.005,0.015] seed 0, detuning 0.002, dt=0.05, 200 steps")


def config_n14() -> TCConfig:
    """n = 14, dim 16384: g as the n = 12 workload (seed 0), 500 steps, renormalise every 50."""
    return TCConfig("n14_precision", 14, draw_couplings(14, 0), 1.002, 1.0, 0.05, 500,
                    renorm_every=50,
                    description="n=14, dim 16384, g~U[0.005,0.015] seed 0, detuning 0.002, dt=0.05, 500 steps, renorm every 50")


def config_n15() -> TCConfig:
    """n = 15, dim 32768 (the paper's largest dimension): g seed 0, precision form only."""
    return TCConfig("n15_precision", 15, draw_couplings(15, 0), 1.002, 1.0, 0.05, 500,
                    renorm_every=50,
                    description="n=15, dim 32768, g~U[0.005,0.015] seed 0, detuning 0.002, dt=0.05, renorm every 50")


def config_n16() -> TCConfig:
    """n = 16, dim 65536 (64 GiB per complex128 matrix): g seed 0, split-BF16 through the host-buffer call."""
    return TCConfig("n16_precision", 16, draw_couplings(16, 0), 1.002, 1.0, 0.05, 500,
                    renorm_every=50,
                    description="n=16, dim 65536, g~U[0.005,0.015] seed 0, detuning 0.002, dt=0.05, renorm every 50")


def config_open(n: int = 14, kappa: float = 0.02) -> TCConfig:
    """Open system (photon leakage at rate kappa): g seed 0, detuning 0.002, dt = 0.05, renorm every 50."""
    return TCConfig("open%d" % n, n, draw_couplings(n, 0), 1.002, 1.0, 0.05, 500, renorm_every=50,
                    description="open system n=%d (excitation blocks k=0..%d), g~U[0.005,0.015] seed 0, "
                                "detuning 0.002, kappa=%g, dt=0.05, renorm every 50" % (n, n, kappa),
                    kappa=kappa)


def config_n11_grad() -> TCConfig:
    """n = 11, dim 2048: g seed 1, 400 steps, loss = excited population of atom 1."""
    return TCConfig("n11_grad", 11, draw_couplings(11, 1), 1.002, 1.0, 0.05, 400,
                    ckpt_every=20, loss_atom=1,
                    description="n=11, dim 2048, g~U[0.005,0.015] seed 1, detuning 0.002, dt=0.05, 400 steps, ckpt 20, loss P_1(T)")


def config_batch(count: int = 64, seed: int = 2, n_lo: int = 6, n_hi: int = 12,
                 steps: int = 200) -> List[TCConfig]:
    """`count` independent systems, n ~ U{n_lo..n_hi}, own g_i; draw order: all n first, then each g."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for j, n in enumerate(ns):
        g = rng.uniform(0.005, 0.015, size=int(n))
        out.append(TCConfig("batch_%d" % j, int(n), g, 1.002, 1.0, 0.05, steps))
    return out


def all_excited_state(n: int) -> np.ndarray:
    """|l_1..l_n = 1..1, 0 photons>: basis index 2^n - 1 (complex128 vector)."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[-1] = 1.0
    return psi


def all_excited_rho(n: int) -> np.ndarray:
    N = 1 << n
    rho = np.zeros((N, N), dtype=np.complex128)
    rho[N - 1, N - 1] = 1.0
    return rho


def random_pure_state(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def random_mixed_state(n: int, rank: int, seed: int):
    """rho = sum_r w_r psi_r psi_r^dag with random w (sum 1) and random psi_r.

    Returns (rho, weights, states) so that a pure-state oracle can propagate
    each component.
    """
    rng = np.random.default_rng(seed)
    N = 1 << n
    w = rng.uniform(0.1, 1.0, size=rank)
    w = w / w.sum()
    states = []
    rho = np.zeros((N, N), dtype=np.complex128)
    for r in range(rank):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        v = v / np.linalg.norm(v)
        states.append(v)
        rho += w[r] * np.outer(v, v.conj())
    return rho, w, states


def random_couplings(n: int, seed: int) -> np.ndarray:
    return draw_couplings(n, seed)
