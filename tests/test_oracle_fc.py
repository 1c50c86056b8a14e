"""Pins for the oracle's FC packing: Theorem 1 by brute force.

Coefficient k < n_o' of i(X) w_j(X) + d_j(X) in Z[X]/(X^N+1) (numpy.convolve
over Python ints) must equal row j*n_o' + k of W I + B (numpy matmul),
including the split case n_i * n_o > N.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth


def _negacyclic_int(a, b):
    N = len(a)
    full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
    out = np.zeros(N, dtype=object)
    out[:] = full[:N]
    out[:len(full) - N] -= full[N:]
    return out


@pytest.mark.parametrize("N,n_in,n_out", [
    (8, 4, 2),        # the paper's n_i = 4, n_o = 2 example
    (64, 8, 8),       # n_i n_o = N
    (64, 5, 3),       # padded with zeros
    (64, 16, 10),     # split: n_o' = 4 rows per polynomial, 3 polynomials
    (64, 6, 20),      # n_i not a power of two: padded to 8 columns
    (256, 64, 10),    # plain-20 FC shape at a small ring
    (128, 64, 100),   # split into 50 blocks of 2 rows
])
def test_theorem1_fc_packing(N, n_in, n_out):
    lay = O.fc_layout(N, n_in, n_out)
    W = synth.ints(N, "W", (n_out, n_in), -128, 127)
    I = synth.ints(N, "I", (n_in,), -8, 7)
    Bv = synth.ints(N, "B", (n_out,), -1000, 1000)
    ref = W @ I + Bv
    ip = O.pack_fc_input(I, lay)
    wp = O.pack_fc_weights(W, lay)
    dp = O.pack_fc_bias(Bv, lay)
    got = []
    for j in range(lay["P"]):
        y = _negacyclic_int(ip, wp[j]) + dp[j]
        got += [int(y[k]) for k in range(lay["rows"][j])]
    assert got == [int(v) for v in ref]
    np.testing.assert_array_equal(O.direct_fc(W, I, Bv), ref)


def test_fc_layout_counts():
    assert O.fc_layout(8192, 64, 10)["P"] == 1
    assert O.fc_layout(4096, 64, 100)["P"] == 2
    assert O.fc_layout(16384, 256, 100)["P"] == 2
    lay = O.fc_layout(16384, 256, 100)
    assert lay["rows"] == [64, 36]


def test_planted_fc_index_mistake_breaks_theorem1():
    N, n_in, n_out = 64, 8, 8
    lay = O.fc_layout(N, n_in, n_out)
    W = synth.ints(9, "W", (n_out, n_in), -128, 127)
    I = synth.ints(9, "I", (n_in,), -8, 7)
    ref = W @ I
    bad = np.zeros((1, N), dtype=np.int64)
    for k in range(n_out):
        bad[0, k] += W[k, 0]
        for l in range(1, n_in):
            bad[0, l * lay["rows_per_poly"] + k] -= W[k, l]      # W_{k,l} instead of W_{k,n_i-l}
    y = _negacyclic_int(O.pack_fc_input(I, lay), bad[0])
    assert [int(y[k]) for k in range(n_out)] != [int(v) for v in ref]
