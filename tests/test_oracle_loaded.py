"""Pins for the oracle's model-load / per-request split (Sec. IV-A: the
server transforms its plaintext polynomials once and stores them).

The "_loaded" layer functions take weights transformed once by the "_load"
functions and must give, word for word, what the definition tier
(schoolbook negacyclic products, no NTT) gives on the untransformed weights:
plain Conv (several groups, both output modes), masked Conv (Alg. 1), plain
FC with P_fc > 1 and a bias, masked FC (Alg. 2).  A planted mistake in the
stored transforms (one word changed) must change the output.
"""

import numpy as np

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537


def _params(N, L):
    ps = O.select_primes(N, L)
    return ps, [O.root_2n(q, N) for q in ps]


def test_conv_loaded_equals_schoolbook_in_both_modes():
    N, L, B = 256, 2, 2
    ps, psis = _params(N, L)
    lay = O.conv_layout(N, 12, 6, 4, 4)
    assert lay["G"] > 1
    cts = synth.residues(81, "ld/ct", (B, lay["G"], 2, L, N), ps)
    F = synth.conv_weights(81, "ld/F", 6, 12, 3, 3, -128, 127)
    wn = O.conv_load(F, ps, psis, lay)
    for mode in (O.OUT_EXTRACTED, O.OUT_PER_CHANNEL):
        want = O.conv_layer(cts, F, ps, psis, lay, mode, tier="schoolbook")
        np.testing.assert_array_equal(O.conv_layer_loaded(cts, wn, ps, psis, lay, mode), want)
    bad = [w.copy() for w in wn]
    bad[1][3, 0, 17] = (int(bad[1][3, 0, 17]) + 1) % ps[1]
    got = O.conv_layer_loaded(cts, bad, ps, psis, lay, O.OUT_PER_CHANNEL)
    assert not np.array_equal(got, O.conv_layer(cts, F, ps, psis, lay, O.OUT_PER_CHANNEL, tier="schoolbook"))


def test_masked_conv_loaded_equals_schoolbook():
    N, L, B = 256, 2, 3
    ps, psis = _params(N, L)
    lay = O.conv_layout(N, 12, 6, 4, 4)
    G, H = lay["G"], lay["H"]
    c0 = synth.residues(82, "ld/c0", (B, G, L, N), ps)
    sh = synth.ints(82, "ld/sh", (B, G, N), 0, T - 1)
    rho = synth.ints(82, "ld/rho", (6, G, N), 0, T - 1)
    shp = synth.ints(82, "ld/shp", (B, H, N), 0, T - 1)
    F = synth.conv_weights(82, "ld/F", 6, 12, 3, 3, -128, 127)
    want = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="schoolbook")
    wn = O.conv_masked_load(F, rho, ps, psis, lay)
    np.testing.assert_array_equal(O.conv_layer_masked_loaded(c0, sh, wn, shp, ps, psis, T, lay), want)


def test_fc_loaded_equals_schoolbook_with_bias_and_several_blocks():
    N, L, B = 128, 2, 2
    ps, psis = _params(N, L)
    lay = O.fc_layout(N, 40, 9)
    assert lay["P"] > 1
    ct = synth.residues(83, "ld/fct", (B, 2, L, N), ps)
    W = synth.fc_weights(83, "ld/W", 9, 40, -128, 127)
    Bv = synth.ints(83, "ld/B", (9,), -500, 500)
    loaded = O.fc_load(W, Bv, ps, psis, lay)
    for mode in (O.OUT_EXTRACTED, O.OUT_PER_CHANNEL):
        want = O.fc_layer(ct, W, Bv, ps, psis, T, lay, mode, tier="schoolbook")
        np.testing.assert_array_equal(O.fc_layer_loaded(ct, loaded, ps, psis, T, lay, mode), want)


def test_masked_fc_loaded_equals_schoolbook():
    N, L, B = 128, 2, 2
    ps, psis = _params(N, L)
    lay = O.fc_layout(N, 40, 9)
    P = lay["P"]
    c0 = synth.residues(84, "ld/mc0", (B, L, N), ps)
    sh = synth.ints(84, "ld/msh", (B, N), 0, T - 1)
    rho = synth.ints(84, "ld/mrho", (P, N), 0, T - 1)
    shp = synth.ints(84, "ld/mshp", (B, P, N), 0, T - 1)
    W = synth.fc_weights(84, "ld/mW", 9, 40, -128, 127)
    Bv = synth.ints(84, "ld/mB", (9,), -500, 500)
    want = O.fc_layer_masked(c0, sh, rho, W, Bv, shp, ps, psis, T, lay, tier="schoolbook")
    loaded = O.fc_masked_load(W, Bv, rho, ps, psis, lay)
    np.testing.assert_array_equal(O.fc_layer_masked_loaded(c0, sh, loaded, shp, ps, psis, T, lay), want)
