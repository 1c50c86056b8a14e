"""Pins for the oracle's NTT tier at the sizes the GPU parity tests use.

The NTT tier is checked against the schoolbook definition word for word
only at N <= 1024 elsewhere.  Here every distinct plain-20 Conv shape at
N = 8192 with 3 limbs (and one wide layer at N = 16384 with 6 limbs) is
checked on 4096 (1024) randomly drawn extracted words, each recomputed by an
O(N) schoolbook dot product, and the FC layer 64 -> 10 at N = 8192 is
checked in full against the schoolbook tier.  A planted mistake in the NTT
tier's product must break the sampled check."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537
PLAIN20_SHAPES = [(3, 16, 32), (16, 16, 32), (16, 32, 32), (32, 32, 16), (32, 64, 16), (64, 64, 8)]


def _ring(N, L):
    ps = O.select_primes(N, L)
    return ps, [O.root_2n(q, N) for q in ps]


def _picks(lay, L, B, count, seed):
    rng = np.random.default_rng(seed)
    N = lay["N"]
    picks = [(int(rng.integers(B)), int(rng.integers(lay["H"])), int(rng.integers(2)), int(rng.integers(L)),
              int(rng.integers(N))) for _ in range(count)]
    # both ends of the polynomial and of the batch, every output polynomial
    picks += [(0, h, 0, 0, 0) for h in range(lay["H"])]
    picks += [(B - 1, lay["H"] - 1, 1, L - 1, N - 1)]
    return picks


def _sampled_check(N, L, ci, co, hw, B, count, seed, tier_out=None):
    ps, psis = _ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    cts = synth.residues(seed, f"fs/ct/{ci}/{co}", (B, lay["G"], 2, L, N), ps)
    F = synth.conv_weights(seed, f"fs/F/{ci}/{co}", co, ci, 3, 3, -128, 127)
    full = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt") if tier_out is None \
        else tier_out(cts, F, ps, psis, lay)
    picks = _picks(lay, L, B, count, seed)
    got = O.conv_layer_sampled(cts, F, ps, lay, picks)
    want = np.array([full[p] for p in picks], dtype=np.uint32)
    return got, want


@pytest.mark.parametrize("ci,co,hw", PLAIN20_SHAPES)
def test_ntt_tier_matches_sampled_schoolbook_on_plain20_shapes(ci, co, hw):
    got, want = _sampled_check(8192, 3, ci, co, hw, 1, 4096, seed=900 + ci + co)
    np.testing.assert_array_equal(got, want)
    assert want.any()


def test_ntt_tier_matches_sampled_schoolbook_on_a_wide_layer():
    # 256 -> 256 at 8x8 on the wide ring: s = 128, G = 2, H = 2
    got, want = _sampled_check(16384, 6, 256, 256, 8, 1, 1024, seed=951)
    np.testing.assert_array_equal(got, want)


def test_fc_ntt_tier_equals_schoolbook_at_full_size():
    N, L = 8192, 3
    ps, psis = _ring(N, L)
    lay = O.fc_layout(N, 64, 10)
    ct = synth.residues(960, "fs/fc/ct", (1, 2, L, N), ps)
    W = synth.fc_weights(960, "fs/fc/W", 10, 64, -128, 127)
    Bv = synth.ints(960, "fs/fc/B", (10,), -1000, 1000)
    a = O.fc_layer(ct, W, Bv, ps, psis, T, lay, O.OUT_EXTRACTED, tier="ntt")
    b = O.fc_layer(ct, W, Bv, ps, psis, T, lay, O.OUT_EXTRACTED, tier="schoolbook")
    np.testing.assert_array_equal(a, b)
    assert a[0, 0, 0, :, :10].any()


def test_planted_ntt_tier_mistake_breaks_the_sampled_check():
    # the NTT tier's output with one output channel's slot class shifted by
    # one position must disagree with the schoolbook samples
    def shifted(cts, F, ps, psis, lay):
        y = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
        s = lay["s"]
        r = lay["off"][0]
        cls = y[:, 0, :, :, r::s].copy()
        y[:, 0, :, :, r::s] = np.roll(cls, 1, axis=-1)
        return y
    got, want = _sampled_check(8192, 3, 16, 16, 32, 1, 4096, seed=916, tier_out=shifted)
    assert not np.array_equal(got, want)
