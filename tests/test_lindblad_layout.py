"""The packed excitation-block layout of the open-system form (host only).

Block k holds the atom strings with popcount(s) <= k; all blocks share one
order of the strings (by popcount, then value), so block k's basis is a
prefix of it.  Checked against the definition written out here.
"""
import math

import pytest


@pytest.mark.parametrize("n", [1, 2, 5, 9, 16])
def test_layout_is_the_definition(n):
    import paper_2403_06937_gb300 as tc
    lay = tc.lindblad_layout(n)
    N = 1 << n
    order = sorted(range(N), key=lambda s: (bin(s).count("1"), s))
    assert lay.basis == order
    dims = [sum(math.comb(n, j) for j in range(k + 1)) for k in range(n + 1)]
    assert lay.dims == dims
    offs = [0]
    for d in dims:
        offs.append(offs[-1] + d * d)
    assert lay.offsets == offs
    # every block's basis is a prefix: the strings of block k are exactly those with popcount <= k
    for k in range(n + 1):
        assert all(bin(s).count("1") <= k for s in order[:dims[k]])
        assert all(bin(s).count("1") > k for s in order[dims[k]:])


def test_layout_rejects_bad_n():
    import paper_2403_06937_gb300 as tc
    with pytest.raises(tc.TCError):
        tc.lindblad_layout(0)
    with pytest.raises(tc.TCError):
        tc.lindblad_layout(17)
