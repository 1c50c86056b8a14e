"""Pins against values the paper prints (tests/golden/).

Table II gives the communication cost of the proposed Conv evaluation for
four plain-20 / ResNet-50 layer shapes at N = 2^13.  Its server -> client
term counts one Q'-bit coefficient per valid output value, w^2 c_o of them
when c_o = c_i.  The oracle's rotation-free extraction (output_slot) must
place exactly that many valid results at distinct (polynomial, slot)
positions that survive extract_conv; combined with the input term, this
count must reproduce the printed megabytes.
"""

from __future__ import annotations

import math
import os

import numpy as np

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2_comm_cost.txt")
N, LOGQ, LOGQP = 8192, 104, 55


def _rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                w, ci, co, mb = line.split()
                out.append((int(w), int(ci), int(co), float(mb)))
    return out


def test_golden_file_has_the_four_table_rows():
    assert [r[:3] for r in _rows()] == [(7, 256, 256), (15, 128, 128), (31, 64, 64), (63, 32, 32)]


def test_valid_output_count_reproduces_table2():
    for w, ci, co, mb in _rows():
        lay = O.conv_layout(N, ci, co, w, w)
        pos = {O.output_slot(lay, n, k, l) for n in range(co) for k in range(w) for l in range(w)}
        # every valid result has its own slot ...
        assert len(pos) == co * w * w
        # ... inside the residue class that extraction keeps for its channel
        for n in (0, co // 2, co - 1):
            hh, slot = O.output_slot(lay, n, w - 1, w - 1)
            assert hh == n // lay["s"] and slot % lay["s"] == lay["off"][n] and slot < N
        bits = N * math.ceil(w * w * ci / N) * LOGQ + len(pos) * LOGQP
        assert round(bits / 8 / 1e6, 2) == mb


def test_extraction_moves_every_valid_value_of_a_small_layer():
    """The same count seen through extract_conv on real data: every valid
    value of every channel arrives in the extracted polynomials."""
    w, ci, co = 4, 8, 8
    lay = O.conv_layout(256, ci, co, w, w)
    rng = np.random.default_rng(0)
    y = rng.integers(1, 1000, size=(co, 256)).astype(np.int64)
    out = O.extract_conv(y, lay)
    for n in range(co):
        for k in range(w):
            for l in range(w):
                hh, slot = O.output_slot(lay, n, k, l)
                assert out[hh, slot] == y[n, slot]
