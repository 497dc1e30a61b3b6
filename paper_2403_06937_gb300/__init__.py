"""Tavis-Cummings unitary evolution on GB300 (arXiv 2403.06937).

Thin torch-facing binding over libtc's C ABI (``include/tc.h``).  Every step of
the computation runs in the library's CUDA kernels; this module only allocates
tensors with torch (device memory, caching allocator, streams) and passes
pointers.  It never computes a result itself and has no CPU path.

    import paper_2403_06937_gb300 as tc
    H = tc.build_hamiltonian(n, g, omega_a, omega_c)
    U = tc.expm(H, n, dt)
    rho, obs = tc.evolve(U, rho0, n, steps, precision="bf16x3", params=p)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _abi
from ._abi import (TC_BF16X3, TC_COUPLING_BOSONIC, TC_COUPLING_QUBIT_PHOTON, TC_FP64, TC_OP_BACKWARD,
                   TC_OP_EVOLVE, TC_OP_EXPM, TC_OP_OBSERVABLES, TC_TF32, TC_TF32X3, TCError)

PRECISIONS = {"fp64": TC_FP64, "bf16x3": TC_BF16X3, "tf32": TC_TF32, "tf32x3": TC_TF32X3,
              "ozaki": _abi.TC_FP64_OZAKI}


@dataclass
class Params:
    """Model parameters of Eq. 4: n atoms, couplings g_1..g_n, frequencies."""
    n: int
    g: Sequence[float]
    omega_a: float = 1.0
    omega_c: float = 1.0
    coupling: int = TC_COUPLING_BOSONIC

    def c(self):
        return _abi.make_params(self.n, self.g, self.omega_a, self.omega_c, self.coupling)


def obs_stride(n: int) -> int:
    return 2 * n + 5


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _work(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def workspace_size(n: int, precision: int = TC_FP64, ops: int = TC_OP_EVOLVE, steps: int = 0,
                   ckpt_every: int = 0) -> int:
    return int(_abi.load().tc_workspace_size(n, precision, ops, steps, ckpt_every))


def device_check() -> None:
    _abi.call("tc_device_check")


def build_hamiltonian(params: Params, device="cuda", stream=None) -> torch.Tensor:
    """tc_build_hamiltonian: dense real H (N x N float64) of Eq. 4."""
    N = 1 << params.n
    H = torch.empty((N, N), dtype=torch.float64, device=device)
    p = params.c()
    _abi.call("tc_build_hamiltonian", ctypes.byref(p), _ptr(H), ctypes.c_void_p(_stream(stream)))
    return H


def expm(H: torch.Tensor, n: int, dt: float, taylor_degree: int = 0, squarings: int = -1, shift: bool = True,
         stream=None, work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """tc_expm: U = e^{-iH dt} (N x N complex128); {10, 0, False} is the paper's Eq. 10."""
    N = 1 << n
    assert H.dtype == torch.float64 and H.is_contiguous() and H.shape == (N, N)
    U = torch.empty((N, N), dtype=torch.complex128, device=H.device)
    need = workspace_size(n, TC_FP64, TC_OP_EXPM)
    if work is None or work.numel() < need:
        work = _work(need, H.device)
    opts = _abi.tc_expm_opts(int(taylor_degree), int(squarings), int(bool(shift)))
    _abi.call("tc_expm", _ptr(H), n, float(dt), ctypes.byref(opts), _ptr(U), _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)))
    return U


def expm_model(params: Params, dt: float, taylor_degree: int = 0, squarings: int = -1, shift: bool = True,
               device="cuda", stream=None, work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """tc_expm_model: U = e^{-iH dt} from the model, H applied as a stencil (no dense H)."""
    n = params.n
    N = 1 << n
    U = torch.empty((N, N), dtype=torch.complex128, device=device)
    need = workspace_size(n, TC_FP64, _abi.TC_OP_EXPM_MODEL)
    if work is None or work.numel() < need:
        work = _work(need, device)
    opts = _abi.tc_expm_opts(int(taylor_degree), int(squarings), int(bool(shift)))
    p = params.c()
    _abi.call("tc_expm_model", ctypes.byref(p), float(dt), ctypes.byref(opts), _ptr(U), _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)))
    return U


def evolve(U: torch.Tensor, rho: torch.Tensor, n: int, steps: int, precision="fp64", renorm_every: int = 0,
           params: Optional[Params] = None, observe: bool = True, inplace: bool = False, stream=None,
           work: Optional[torch.Tensor] = None):
    """tc_evolve: `steps` steps of rho <- U rho U^dag.  Returns (rho_T, obs or None)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    N = 1 << n
    assert U.dtype == torch.complex128 and U.is_contiguous() and U.shape == (N, N)
    assert rho.dtype == torch.complex128 and rho.is_contiguous() and rho.shape == (N, N)
    out = rho if inplace else rho.clone()
    obs = torch.empty((steps + 1, obs_stride(n)), dtype=torch.float64, device=rho.device) if observe else None
    need = workspace_size(n, prec, TC_OP_EVOLVE)
    if work is None or work.numel() < need:
        work = _work(need, rho.device)
    p = params.c() if params is not None else None
    _abi.call("tc_evolve", _ptr(U), _ptr(out), n, int(steps), prec, int(renorm_every),
              ctypes.byref(p) if p is not None else None, _ptr(obs), _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)))
    return out, obs


@dataclass
class LindbladLayout:
    """Packed excitation-block layout of the open-system form (tc_lindblad_layout)."""
    n: int
    dims: list        # d_k, k = 0..n
    offsets: list     # element offset of block k; offsets[n + 1] = total
    basis: list       # atom string at each block position

    @property
    def total(self) -> int:
        return self.offsets[-1]

    def blocks(self, packed: torch.Tensor):
        """Views [d_k x d_k] of a packed state, k = 0..n."""
        return [packed[self.offsets[k]:self.offsets[k + 1]].view(self.dims[k], self.dims[k])
                for k in range(self.n + 1)]


def lindblad_layout(n: int) -> LindbladLayout:
    dims = (ctypes.c_int * (n + 1))()
    offs = (ctypes.c_size_t * (n + 2))()
    basis = (ctypes.c_int * (1 << n))()
    _abi.call("tc_lindblad_layout", int(n), ctypes.cast(dims, ctypes.c_void_p), ctypes.cast(offs, ctypes.c_void_p),
              ctypes.cast(basis, ctypes.c_void_p))
    return LindbladLayout(n, list(dims), [int(o) for o in offs], list(basis))


def lindblad_propagators(params: Params, dt: float, device="cuda", stream=None,
                         work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """tc_lindblad_propagators: packed U_k = e^{-i H_k dt} for every excitation block."""
    lay = lindblad_layout(params.n)
    U = torch.empty(lay.total, dtype=torch.complex128, device=device)
    need = workspace_size(params.n, TC_FP64, _abi.TC_OP_LINDBLAD)
    if work is None or work.numel() < need:
        work = _work(need, device)
    p = params.c()
    _abi.call("tc_lindblad_propagators", ctypes.byref(p), float(dt), _ptr(U), _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)))
    return U


def lindblad_evolve(params: Params, kappa: float, dt: float, U: torch.Tensor, rho: torch.Tensor, steps: int,
                    precision="fp64", renorm_every: int = 0, observe: bool = True, inplace: bool = False,
                    stream=None, work: Optional[torch.Tensor] = None):
    """tc_lindblad_evolve: `steps` split steps of Eq. 5 with photon leakage.  Returns (rho_T, obs or None)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    n = params.n
    lay = lindblad_layout(n)
    for t in (U, rho):
        assert t.dtype == torch.complex128 and t.is_contiguous() and t.numel() == lay.total
    out = rho if inplace else rho.clone()
    obs = torch.empty((steps + 1, obs_stride(n)), dtype=torch.float64, device=rho.device) if observe else None
    need = workspace_size(n, prec, _abi.TC_OP_LINDBLAD)
    if work is None or work.numel() < need:
        work = _work(need, rho.device)
    p = params.c()
    _abi.call("tc_lindblad_evolve", ctypes.byref(p), float(kappa), float(dt), _ptr(U), _ptr(out), int(steps), prec,
              int(renorm_every), _ptr(obs), _ptr(work), work.numel(), ctypes.c_void_p(_stream(stream)))
    return out, obs


def observables(rho: torch.Tensor, n: int, params: Optional[Params] = None, stream=None) -> torch.Tensor:
    """tc_observables: [P_1..P_n, <p>, P(0..n), Tr rho, Tr rho^2, E] of a density matrix."""
    N = 1 << n
    assert rho.dtype == torch.complex128 and rho.is_contiguous() and rho.shape == (N, N)
    out = torch.empty(obs_stride(n), dtype=torch.float64, device=rho.device)
    work = _work(workspace_size(n, TC_FP64, TC_OP_OBSERVABLES), rho.device)
    p = params.c() if params is not None else None
    _abi.call("tc_observables", _ptr(rho), n, ctypes.byref(p) if p is not None else None, _ptr(out), _ptr(work),
              work.numel(), ctypes.c_void_p(_stream(stream)))
    return out


def expectation_diag(rho: torch.Tensor, n: int, O_diag: torch.Tensor, stream=None) -> torch.Tensor:
    """tc_expectation_diag: Tr(diag(O) rho) as a 0-d float64 tensor on rho's device."""
    N = 1 << n
    assert rho.dtype == torch.complex128 and rho.is_contiguous() and rho.shape == (N, N)
    assert O_diag.dtype == torch.float64 and O_diag.is_contiguous() and O_diag.numel() == N
    out = torch.empty((), dtype=torch.float64, device=rho.device)
    _abi.call("tc_expectation_diag", _ptr(rho), n, _ptr(O_diag), _ptr(out), ctypes.c_void_p(_stream(stream)))
    return out


def evolve_host(U: torch.Tensor, rho_host: torch.Tensor, n: int, steps: int, precision="fp64",
                renorm_every: int = 0, params: Optional[Params] = None, obs_host: Optional[torch.Tensor] = None,
                stream=None, work: Optional[torch.Tensor] = None) -> None:
    """tc_evolve_host: rho_host (CPU complex128, ideally pinned) stepped in place on the GPU; blocks."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    N = 1 << n
    assert rho_host.device.type == "cpu" and rho_host.dtype == torch.complex128 and rho_host.shape == (N, N)
    # a page-locked buffer lets the pipelined tensor-core forms skip the device copy of rho
    op = _abi.TC_OP_EVOLVE_HOST_PINNED if rho_host.is_pinned() else _abi.TC_OP_EVOLVE_HOST
    need = workspace_size(n, prec, op, steps)
    if work is None or work.numel() < need:
        work = _work(need, U.device)
    p = params.c() if params is not None else None
    _abi.call("tc_evolve_host", _ptr(U), _ptr(rho_host), n, int(steps), prec, int(renorm_every),
              ctypes.byref(p) if p is not None else None, _ptr(obs_host), _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)))


def evolve_backward(params: Params, dt: float, steps: int, rho0: torch.Tensor, U: torch.Tensor,
                    O_diag: torch.Tensor, ckpt_every: int = 20, precision="fp64", stream=None,
                    work: Optional[torch.Tensor] = None):
    """tc_evolve_backward: (grad, loss) of L = Tr(diag(O) rho_K) w.r.t. (g_1..g_n, omega_a, omega_c).

    grad is a float64 numpy-convertible CPU tensor of n + 2 values; the call blocks.
    """
    n = params.n
    N = 1 << n
    assert rho0.dtype == torch.complex128 and rho0.is_contiguous() and rho0.shape == (N, N)
    assert U.dtype == torch.complex128 and U.is_contiguous() and U.shape == (N, N)
    assert O_diag.dtype == torch.float64 and O_diag.is_cuda and O_diag.numel() == N
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    need = workspace_size(n, prec, TC_OP_BACKWARD, steps, ckpt_every)
    if work is None or work.numel() < need:
        work = _work(need, rho0.device)
    grad = (ctypes.c_double * (n + 2))()
    loss = ctypes.c_double()
    p = params.c()
    _abi.call("tc_evolve_backward", ctypes.byref(p), float(dt), int(steps), _ptr(rho0), _ptr(U), int(ckpt_every),
              prec, _ptr(O_diag.contiguous()), grad, ctypes.byref(loss), _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)))
    return torch.tensor(list(grad), dtype=torch.float64), float(loss.value)


class EvolveFn(torch.autograd.Function):
    """L = Tr(diag(O) rho_K) as a differentiable function of (g, omega_a, omega_c).

    forward: H (Eq. 4), U = e^{-iH dt} (tc_expm), K steps of rho <- U rho U^dag
    (tc_evolve) and L (tc_expectation_diag); nothing of the reverse pass runs.
    backward (only when a gradient is asked for): tc_evolve_backward, the
    reverse mode with checkpoints every `ckpt_every` steps.
    precision: "fp64" (DMMA products) or "ozaki" (the products emulated at FP64
    accuracy on the BF16 tensor cores; n >= 7), for both passes.
    Inputs g (n,), omega_a (), omega_c () are float64 tensors; rho0 and O_diag
    are CUDA tensors.  Returns a 0-d float64 tensor on rho0's device.
    """

    @staticmethod
    def forward(ctx, g, omega_a, omega_c, rho0, O_diag, dt, steps, ckpt_every=20, coupling=TC_COUPLING_BOSONIC,
                precision="fp64"):
        if precision not in ("fp64", "ozaki"):
            raise ValueError("EvolveFn: precision must be 'fp64' or 'ozaki'")
        n = int(g.numel())
        params = Params(n, [float(x) for x in g.detach().cpu()], float(omega_a), float(omega_c), coupling)
        U = expm(build_hamiltonian(params, device=rho0.device), n, dt)
        rho, _ = evolve(U, rho0, n, steps, precision, params=params, observe=False)
        O = O_diag.contiguous()
        loss = expectation_diag(rho, n, O)
        ctx.save_for_backward(rho0, O, U)
        ctx.params, ctx.dt, ctx.steps, ctx.ckpt_every, ctx.precision = params, dt, steps, ckpt_every, precision
        ctx.devices = (g.device, omega_a.device if torch.is_tensor(omega_a) else g.device,
                       omega_c.device if torch.is_tensor(omega_c) else g.device)
        return loss

    @staticmethod
    def backward(ctx, gout):
        none = (None,) * 7
        if not any(ctx.needs_input_grad[:3]):
            return (None, None, None) + none
        rho0, O, U = ctx.saved_tensors
        grad, _ = evolve_backward(ctx.params, ctx.dt, ctx.steps, rho0, U, O, ctx.ckpt_every,
                                  precision=ctx.precision)
        n = ctx.params.n
        scale = gout.detach().to("cpu", torch.float64)
        dg, dwa, dwc = grad[:n] * scale, grad[n] * scale, grad[n + 1] * scale
        return (dg.to(ctx.devices[0]), dwa.to(ctx.devices[1]), dwc.to(ctx.devices[2])) + none


def batch_evolve(Us, rhos, steps: int, precision="bf16x3", renorm_every: int = 0, params=None,
                 observe: bool = True, inplace: bool = False, stream=None, work: Optional[torch.Tensor] = None):
    """tc_batch_evolve: step many systems of uneven size together.

    Us, rhos: lists of (N_b x N_b) complex128 CUDA tensors; params: list of
    Params or None.  Returns (list of rho_T, list of obs or None).
    """
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    count = len(Us)
    ns = []
    for U, r in zip(Us, rhos):
        N = U.shape[0]
        n = N.bit_length() - 1
        assert 1 << n == N and U.dtype == torch.complex128 and r.shape == U.shape and r.dtype == torch.complex128
        ns.append(n)
    outs = rhos if inplace else [r.clone() for r in rhos]
    obs = [torch.empty((steps + 1, obs_stride(n)), dtype=torch.float64, device=r.device) for n, r in zip(ns, rhos)] \
        if observe else None
    n_arr = (ctypes.c_int * count)(*ns)
    need = int(_abi.load().tc_batch_workspace_size(count, n_arr, prec))
    if work is None or work.numel() < need:
        work = _work(need, rhos[0].device)
    U_arr = (ctypes.c_void_p * count)(*[U.data_ptr() for U in Us])
    R_arr = (ctypes.c_void_p * count)(*[r.data_ptr() for r in outs])
    O_arr = (ctypes.c_void_p * count)(*[o.data_ptr() for o in obs]) if observe else None
    P_arr = None
    keep = []
    if params is not None:
        cps = [p.c() for p in params]
        keep = cps
        P_arr = (_abi.tc_params * count)(*cps)
    _abi.call("tc_batch_evolve", count, n_arr, U_arr, R_arr, int(steps), prec, int(renorm_every), P_arr, O_arr,
              _ptr(work), work.numel(), ctypes.c_void_p(_stream(stream)))
    del keep
    return outs, obs


def autotune(n: int, precision="bf16x3", stream=None, work: Optional[torch.Tensor] = None):
    """tc_autotune: time the built kernel configurations for (n, precision); returns the choice."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    need = workspace_size(n, prec, TC_OP_EVOLVE)
    if work is None or work.numel() < need:
        work = _work(need, "cuda")
    out = (ctypes.c_int * 4)()
    _abi.call("tc_autotune", n, prec, _ptr(work), work.numel(), ctypes.c_void_p(_stream(stream)), out)
    return {"f64_tile": out[0], "tc_group": out[1], "tc_stages": out[2], "tc_shape": out[3]}


def autotune_lookup(n: int, precision="bf16x3"):
    """tc_autotune_lookup: the configuration in use for (n, precision) (host only)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    out = (ctypes.c_int * 4)()
    _abi.call("tc_autotune_lookup", n, prec, out)
    return {"f64_tile": out[0], "tc_group": out[1], "tc_stages": out[2], "tc_shape": out[3]}


# tile shapes of the tensor-core products (tc_autotune_set's tc_shape)
TILE_SHAPES = {"auto": 0, "single": 1, "pair32": 2, "pair_wide": 3}


def autotune_set(n: int, precision="bf16x3", f64_tile: int = 32, tc_group: int = 8, tc_stages: int = 0,
                 tc_shape=0) -> None:
    """tc_autotune_set: pin the configuration for (n, precision) in this process."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if prec != TC_FP64 and tc_stages == 0:
        tc_stages = {TC_BF16X3: 4, TC_TF32X3: 6, TC_TF32: 8}[prec]
    shape = TILE_SHAPES[tc_shape] if isinstance(tc_shape, str) else int(tc_shape)
    arr = (ctypes.c_int * 4)(int(f64_tile), int(tc_group), int(tc_stages), shape)
    _abi.call("tc_autotune_set", n, prec, arr)


def batch_autotune(ns, precision="bf16x3", stream=None, work: Optional[torch.Tensor] = None):
    """tc_batch_autotune: tile shape and raster group for batches of this composition; returns the choice."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    count = len(ns)
    n_arr = (ctypes.c_int * count)(*[int(x) for x in ns])
    need = int(_abi.load().tc_batch_workspace_size(count, n_arr, prec))
    if work is None or work.numel() < need:
        work = _work(need, "cuda")
    out = (ctypes.c_int * 2)()
    _abi.call("tc_batch_autotune", count, n_arr, prec, _ptr(work), work.numel(),
              ctypes.c_void_p(_stream(stream)), out)
    return {"tc_group": out[0], "tc_shape": out[1]}


def batch_autotune_set(ns, precision="bf16x3", tc_group: int = 8, tc_shape=0) -> None:
    """tc_batch_autotune_set: pin the batch tile shape and raster group for this composition in this process."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    count = len(ns)
    n_arr = (ctypes.c_int * count)(*[int(x) for x in ns])
    shape = TILE_SHAPES[tc_shape] if isinstance(tc_shape, str) else int(tc_shape)
    arr = (ctypes.c_int * 2)(int(tc_group), shape)
    _abi.call("tc_batch_autotune_set", count, n_arr, prec, arr)


def batch_autotune_lookup(ns, precision="bf16x3"):
    """tc_batch_autotune_lookup: the batch choice for this composition, or None (host only)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    count = len(ns)
    n_arr = (ctypes.c_int * count)(*[int(x) for x in ns])
    out = (ctypes.c_int * 2)()
    found = ctypes.c_int(0)
    _abi.call("tc_batch_autotune_lookup", count, n_arr, prec, out, ctypes.byref(found))
    return {"tc_group": out[0], "tc_shape": out[1]} if found.value else None


def launch_count() -> int:
    """Kernels launched by libtc in this process."""
    return int(_abi.load().tc_launch_count())


def timing_enable(on: bool = True) -> None:
    _abi.call("tc_timing_enable", int(bool(on)))


def timing_read():
    """(launches, device ms, FLOPs) of the product kernels timed since the last read."""
    L = ctypes.c_longlong()
    ms = ctypes.c_double()
    fl = ctypes.c_double()
    _abi.call("tc_timing_read", ctypes.byref(L), ctypes.byref(ms), ctypes.byref(fl))
    return int(L.value), float(ms.value), float(fl.value)


def phases_enable(on: bool = True) -> None:
    """tc_phases_enable: record event marks at the phase boundaries of tc_evolve_host calls."""
    _abi.call("tc_phases_enable", int(bool(on)))


def phases_read(max_marks: int = 64):
    """tc_phases_read: [(mark name, ms after the first mark)] recorded since the last read."""
    ms = (ctypes.c_double * max_marks)()
    names = ctypes.create_string_buffer(16 * max_marks + 1)
    count = ctypes.c_int()
    _abi.call("tc_phases_read", ms, names, len(names), int(max_marks), ctypes.byref(count))
    got = names.value.decode().split("\n")[:min(count.value, max_marks)]
    return [(nm, float(ms[i])) for i, nm in enumerate(got)]


def sync_status(stream=None) -> None:
    _abi.call("tc_sync_status", ctypes.c_void_p(_stream(stream)))


__all__ = ["Params", "TCError", "build_hamiltonian", "expm", "expm_model", "evolve", "LindbladLayout",
           "lindblad_layout", "lindblad_propagators", "lindblad_evolve", "evolve_host", "observables",
           "expectation_diag",
           "evolve_backward", "EvolveFn", "batch_evolve", "autotune", "autotune_lookup", "autotune_set", "batch_autotune", "batch_autotune_set", "batch_autotune_lookup",
           "workspace_size", "launch_count", "timing_enable", "timing_read", "phases_enable", "phases_read",
           "device_check", "sync_status", "obs_stride", "PRECISIONS", "TC_FP64", "TC_BF16X3", "TC_TF32",
           "TC_TF32X3", "TC_COUPLING_BOSONIC", "TC_COUPLING_QUBIT_PHOTON", "TC_OP_EXPM", "TC_OP_EVOLVE",
           "TC_OP_OBSERVABLES", "TC_OP_BACKWARD"]
