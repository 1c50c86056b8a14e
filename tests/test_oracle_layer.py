"""Pins for the oracle's server step and its RLWE checks.

* decrypt(encrypt(m)) = m (secret- and public-key forms, 1 and 3 limbs);
* the full single-Conv-layer check: Enc(I) -> server Conv (per-channel
  products) -> decrypt -> the output slots equal the plaintext convolution
  mod t.  With a ternary secret and centered-binomial (eta = 3) error the
  noise after the product is at most 3 * ||f||_1 < Delta/2, so this holds
  with certainty, not with high probability;
* a trivial ciphertext (c1 = 0) through the extracted output decrypts to the
  convolution at every valid slot;
* the same for FC layers (Theorem 1 through encryption), bias included;
* the schoolbook tier and the NTT tier agree word for word, and sampled
  coefficients agree with both.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537


def _params(N, L):
    ps = O.select_primes(N, L)
    return ps, [O.root_2n(q, N) for q in ps]


@pytest.mark.parametrize("N,L", [(16, 1), (64, 1), (64, 3)])
def test_encrypt_decrypt_round_trip(N, L):
    ps, _ = _params(N, L)
    Q = int(np.prod([int(q) for q in ps], dtype=object))
    # BFV with Delta = floor(Q/t) decrypts m exactly while
    # |m| (Q mod t)/Q + t |noise| / Q < 1/2; one 30-bit limb leaves room for
    # |m| up to a few thousand, three limbs for the whole range mod t.
    mmax = T // 2 if L > 1 else 2048
    assert mmax * (Q % T) / Q + T * (3 + 3 * N) / Q < 0.5
    m = synth.ints(N, "m", (N,), -mmax, mmax)
    s = synth.ternary(N, "s", N)
    a = synth.residues(N, "a", (L, N), ps)
    e = synth.cbd(N, "e", N, 3)
    ct = O.encrypt_sk(m, s, a, e, ps, T)
    np.testing.assert_array_equal(O.decrypt(ct, s, ps, T), m)
    v, e0, e1 = synth.v_poly(N, "v", N), synth.cbd(N, "e0", N), synth.cbd(N, "e1", N)
    ct = O.encrypt_pk(m, s, a, e, v, e0, e1, ps, T)
    np.testing.assert_array_equal(O.decrypt(ct, s, ps, T), m)


def _encrypt_groups(ip, s, ps, seed):
    G, N = ip.shape
    out = np.zeros((1, G, 2, len(ps), N), dtype=np.uint32)
    for g in range(G):
        a = synth.residues(seed, f"a{g}", (len(ps), N), ps)
        e = synth.cbd(seed, f"e{g}", N, 3)
        out[0, g] = O.encrypt_sk(ip[g], s, a, e, ps, T)
    return out


@pytest.mark.slow
def test_single_conv_layer_encrypt_eval_decrypt_equals_convolution():
    """The single 3x3 Conv config: N = 2048, one 30-bit prime, t = 65537,
    input 3x16x16 and weights in [-8, 7], 4 output channels, same padding."""
    N, ci, co, h, w = 2048, 3, 4, 16, 16
    ps, psis = _params(N, 1)
    lay = O.conv_layout(N, ci, co, h, w)
    I = synth.ints(1, "conv1/I", (ci, h, w), -8, 7)
    F = synth.ints(1, "conv1/F", (co, ci, 3, 3), -8, 7)
    s = synth.ternary(1, "conv1/s", N)
    cts = _encrypt_groups(O.pack_input(I, lay), s, ps, seed=1)
    y = O.conv_layer(cts, F, ps, psis, lay, mode=O.OUT_PER_CHANNEL)
    ref = O.centered(O.direct_conv(I, F, 1), T)
    for n in range(co):
        m = O.decrypt(y[0, n], s, ps, T)
        for k in range(lay["h_out"]):
            for l in range(lay["w_out"]):
                assert m[O.output_slot(lay, n, k, l)[1]] == ref[n, k, l]
    # extracted output of a trivial ciphertext (c1 = 0): c0 = Delta*i + e
    triv = cts.copy()
    for g in range(lay["G"]):
        e = synth.cbd(1, f"t{g}", N, 3)
        triv[0, g, 0, 0] = O.encrypt_sk(O.pack_input(I, lay)[g], np.zeros(N, np.int64),
                                        np.zeros((1, N), np.uint32), e, ps, T)[0, 0]
        triv[0, g, 1] = 0
    out = O.conv_layer(triv, F, ps, psis, lay, mode=O.OUT_EXTRACTED)
    zero_s = np.zeros(N, np.int64)
    for hh in range(lay["H"]):
        m = O.decrypt(out[0, hh], zero_s, ps, T)
        for n in range(co):
            if n // lay["s"] != hh:
                continue
            for k in range(lay["h_out"]):
                for l in range(lay["w_out"]):
                    assert m[O.output_slot(lay, n, k, l)[1]] == ref[n, k, l]


def test_multi_limb_conv_decrypts_through_crt():
    N, ci, co, h, w = 256, 5, 6, 4, 4
    ps, psis = _params(N, 3)
    lay = O.conv_layout(N, ci, co, h, w)
    assert lay["G"] > 1
    I = synth.ints(2, "I", (ci, h, w), -8, 7)
    F = synth.ints(2, "F", (co, ci, 3, 3), -128, 127)
    s = synth.ternary(2, "s", N)
    cts = _encrypt_groups(O.pack_input(I, lay), s, ps, seed=2)
    y = O.conv_layer(cts, F, ps, psis, lay, mode=O.OUT_PER_CHANNEL)
    ref = O.centered(O.direct_conv(I, F, 1), T)
    for n in range(co):
        m = O.decrypt(y[0, n], s, ps, T)
        got = np.array([[m[O.output_slot(lay, n, k, l)[1]] for l in range(w)] for k in range(h)])
        np.testing.assert_array_equal(got, ref[n])


def test_fc_layer_encrypt_eval_decrypt_equals_wi_plus_b():
    N, n_in, n_out = 256, 64, 10
    ps, psis = _params(N, 2)
    lay = O.fc_layout(N, n_in, n_out)
    W = synth.ints(3, "W", (n_out, n_in), -128, 127)
    I = synth.ints(3, "I", (n_in,), -8, 7)
    Bv = synth.ints(3, "B", (n_out,), -500, 500)
    s = synth.ternary(3, "s", N)
    a = synth.residues(3, "a", (2, N), ps)
    ct = O.encrypt_sk(O.pack_fc_input(I, lay), s, a, synth.cbd(3, "e", N), ps, T)[None]
    y = O.fc_layer(ct, W, Bv, ps, psis, T, lay, mode=O.OUT_PER_CHANNEL)
    ref = O.centered(W @ I + Bv, T)
    got = []
    for j in range(lay["P"]):
        m = O.decrypt(y[0, j], s, ps, T)
        got += list(m[:lay["rows"][j]])
    np.testing.assert_array_equal(np.array(got), ref)
    ye = O.fc_layer(ct, W, Bv, ps, psis, T, lay, mode=O.OUT_EXTRACTED)
    for j in range(lay["P"]):
        np.testing.assert_array_equal(ye[0, j, :, :, :lay["rows"][j]], y[0, j, :, :, :lay["rows"][j]])
        assert not ye[0, j, :, :, lay["rows"][j]:].any()


@pytest.mark.parametrize("N,L,ci,co,hw,B", [(256, 2, 5, 6, 4, 1), (1024, 1, 16, 8, 8, 2),
                                            (512, 3, 3, 4, 8, 1)])
def test_schoolbook_and_ntt_tiers_agree(N, L, ci, co, hw, B):
    ps, psis = _params(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    cts = synth.residues(N, "ct", (B, lay["G"], 2, L, N), ps)
    F = synth.ints(N, "F", (co, ci, 3, 3), -128, 127)
    for mode in (O.OUT_EXTRACTED, O.OUT_PER_CHANNEL):
        a = O.conv_layer(cts, F, ps, psis, lay, mode, tier="schoolbook")
        b = O.conv_layer(cts, F, ps, psis, lay, mode, tier="ntt")
        np.testing.assert_array_equal(a, b)
    picks = [(0, 0, 0, 0, 0), (B - 1, lay["H"] - 1, 1, L - 1, N - 1), (0, 0, 1, 0, 5),
             (0, lay["H"] - 1, 0, L - 1, lay["s"] * 3 + 1)]
    got = O.conv_layer_sampled(cts, F, ps, lay, picks)
    full = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
    np.testing.assert_array_equal(got, np.array([full[p] for p in picks], dtype=np.uint32))


def test_fc_tiers_agree():
    N, L = 512, 2
    ps, psis = _params(N, L)
    lay = O.fc_layout(N, 64, 20)
    ct = synth.residues(4, "ct", (2, 2, L, N), ps)
    W = synth.ints(4, "W", (20, 64), -128, 127)
    Bv = synth.ints(4, "B", (20,), -9, 9)
    for mode in (O.OUT_EXTRACTED, O.OUT_PER_CHANNEL):
        np.testing.assert_array_equal(
            O.fc_layer(ct, W, Bv, ps, psis, T, lay, mode, tier="schoolbook"),
            O.fc_layer(ct, W, Bv, ps, psis, T, lay, mode, tier="ntt"))
