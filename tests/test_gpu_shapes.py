"""Tile shapes of the tensor-core products (the autotuner's choice): one CTA
per 128 x 128 tile, CTA pairs on the 2-SM MMA with 32-byte K rows, or CTA
pairs with wide K rows.  Every shape accumulates each output element in the
same order (K slice by K slice, the part products in one fixed order) and
ends in the same epilogue, so the shape changes speed, not bits: the
single-system step, the batched step (power-of-two tile counts, and one-tile
systems whose odd CTA has no rows) and the open-system blocks (odd tile
counts) give bitwise equal results in every shape."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = ["single", "pair32", "pair_wide"]


@pytest.fixture(scope="module")
def tc():
    from paper_2403_06937_gb300 import build
    build.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    return tc


def _pinned(tc, n, precision, shape):
    c = tc.autotune_lookup(n, precision)
    tc.autotune_set(n, precision, c["f64_tile"], c["tc_group"], c["tc_stages"], shape)


def _runs(tc, ns, precisions, fn):
    out = {}
    for n in ns:
        for prec in precisions:
            saved = tc.autotune_lookup(n, prec)
            try:
                for shape in SHAPES:
                    _pinned(tc, n, prec, shape)
                    out[(n, prec, shape)] = fn(n, prec)
            finally:
                tc.autotune_set(n, prec, saved["f64_tile"], saved["tc_group"], saved["tc_stages"],
                                saved["tc_shape"])
    return out


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_single_system_shapes_give_the_same_bits(tc, precision):
    n = 10   # 8 x 8 tiles
    g = W.draw_couplings(n, 4) * 4
    p = tc.Params(n, list(g), 1.01, 1.0)
    U = tc.expm(tc.build_hamiltonian(p), n, 0.1)
    rho0, _, _ = W.random_mixed_state(n, 3, 5)
    r0 = torch.from_numpy(rho0).cuda()
    res = _runs(tc, [n], [precision], lambda n_, pr: tc.evolve(U, r0, n_, 4, pr, params=p))
    ref = res[(n, precision, "single")]
    for shape in SHAPES[1:]:
        assert _same(ref, res[(n, precision, shape)]), shape


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "tf32"])
def test_batch_shapes_give_the_same_bits(tc, precision):
    ns = [3, 9, 6, 7, 8, 9, 5, 7]   # 1, 2 and 4 tiles a side
    rng = np.random.default_rng(3)
    sys_ = []
    for k, n in enumerate(ns):
        g = rng.uniform(0.005, 0.015, size=n) * 6
        p = tc.Params(n, list(map(float, g)), 1.002, 1.0)
        U = tc.expm(tc.build_hamiltonian(p), n, 0.05)
        rho, _, _ = W.random_mixed_state(n, min(3, 1 << n), 200 + k)
        sys_.append((p, U, torch.from_numpy(rho).cuda()))

    def run(n_, pr):
        rhos, obs = tc.batch_evolve([s[1] for s in sys_], [s[2] for s in sys_], 4, pr,
                                    params=[s[0] for s in sys_])
        tc.sync_status()
        return rhos + obs

    res = _runs(tc, [max(ns)], [precision], run)
    ref = res[(max(ns), precision, "single")]
    for shape in SHAPES[1:]:
        assert _same(ref, res[(max(ns), precision, shape)]), shape
    # and each system equals its standalone run
    for (p, U, r0), rb in zip(sys_, ref[:len(ns)]):
        ra, _ = tc.evolve(U, r0, p.n, 4, precision, params=p)
        assert torch.equal(ra, rb), p.n


@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
def test_open_system_block_shapes_give_the_same_bits(tc, precision):
    """n = 9: excitation blocks of 1 to 4 tiles a side, some of them odd (the
    odd CTA of the last row pair has no rows), kappa = 0.05, 3 steps."""
    n = 9
    g = W.draw_couplings(n, 6) * 4
    p = tc.Params(n, list(g), 1.002, 1.0)
    dt = 0.05
    U = tc.lindblad_propagators(p, dt)
    lay = tc.lindblad_layout(n)
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    rng = np.random.default_rng(11)
    dims = [blk.shape[0] for blk in lay.blocks(rho)]
    assert any(-(-d // 128) % 2 == 1 and d > 128 for d in dims)   # an odd tile count above one
    for blk in lay.blocks(rho):
        d = blk.shape[0]
        A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        M = A @ A.conj().T
        blk.copy_(torch.from_numpy(M / np.trace(M).real / (n + 1)))

    def run(n_, pr):
        out, obs = tc.lindblad_evolve(p, 0.05, dt, U, rho, 3, pr)
        tc.sync_status()
        return [out, obs]

    res = _runs(tc, [n], [precision], run)
    ref = res[(n, precision, "single")]
    for shape in SHAPES[1:]:
        assert _same(ref, res[(n, precision, shape)]), shape


def test_batch_autotune_keeps_the_bits(tc):
    """tc_batch_autotune picks a built shape and group for the batch's
    composition, and the batch run in it gives the same bits."""
    ns = [3, 9, 6, 7, 8, 9, 5, 7]
    rng = np.random.default_rng(5)
    Us, rhos, ps = [], [], []
    for k, n in enumerate(ns):
        g = rng.uniform(0.005, 0.015, size=n) * 6
        p = tc.Params(n, list(map(float, g)), 1.002, 1.0)
        Us.append(tc.expm(tc.build_hamiltonian(p), n, 0.05))
        rho, _, _ = W.random_mixed_state(n, min(3, 1 << n), 300 + k)
        rhos.append(torch.from_numpy(rho).cuda())
        ps.append(p)
    before, ob = tc.batch_evolve(Us, rhos, 3, "bf16x3", params=ps)
    choice = tc.batch_autotune(ns, "bf16x3")
    assert choice["tc_shape"] in (1, 2, 3) and choice["tc_group"] in (4, 8, 12, 16)
    after, oa = tc.batch_evolve(Us, rhos, 3, "bf16x3", params=ps)
    tc.sync_status()
    assert _same(before, after) and _same(ob, oa)
