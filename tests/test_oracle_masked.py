"""Pins for the oracle's whole Conv protocol (Alg. 1): the masked server
step, the client's c1 share and the key-free decode.

* Noiseless identity: with every error polynomial 0, the server's c0^r and
  the client's c1^r add up to Delta_Q (extract(i * fhat) + sh') modulo every
  prime, exactly (the v rho b and sh fhat terms cancel).  The right-hand
  side is built from the packing, the schoolbook product and the
  extraction, which are pinned on their own elsewhere.
* The identity fails when the server drops its share term, when the
  client drops its mask term, or when the mask term's sign is flipped: each
  term is needed and has the sign the reading gives it.
* With RLWE noise (public-key encryption, centered-binomial errors) the
  decode of c0^r + c1^r minus sh' is the plaintext convolution mod t at every
  valid slot (3 limbs leave Delta_Q / 2 far above the noise).
* The schoolbook and NTT tiers of the masked server step agree.
"""

import numpy as np

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537


def _params(N, L):
    ps = O.select_primes(N, L)
    return ps, [O.root_2n(q, N) for q in ps]


def _case(N, L, ci, co, hw, seed, noise):
    ps, psis = _params(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    G, H = lay["G"], lay["H"]
    I = synth.ints(seed, "mk/I", (ci, hw, hw), -8, 7)
    F = synth.ints(seed, "mk/F", (co, ci, 3, 3), -128, 127)
    ip = O.pack_input(I, lay)                                     # [G][N] packed input
    sh = synth.ints(seed, "mk/sh", (1, G, N), 0, T - 1)           # server's share of the input
    rho = synth.ints(seed, "mk/rho", (co, G, N), 0, T - 1)
    shp = synth.ints(seed, "mk/shp", (1, H, N), 0, T - 1)         # share added to the output
    s = synth.ternary(seed, "mk/s", N)
    a = synth.residues(seed, "mk/a", (L, N), ps)
    z = np.zeros(N, np.int64)
    e = synth.cbd(seed, "mk/e", N) if noise else z
    b_pk = np.zeros((L, N), np.uint32)
    for l, q in enumerate(ps):
        b_pk[l] = ((-O.negacyclic_mul(a[l], O.to_residues(s, q), q).astype(np.int64) + e) % q).astype(np.uint32)
    ish = ip + sh[0]                                              # what the client holds
    c0 = np.zeros((1, G, L, N), np.uint32)
    v = np.zeros((G, N), np.int64)
    for g in range(G):
        v[g] = synth.v_poly(seed, f"mk/v{g}", N)
        e0 = synth.cbd(seed, f"mk/e0{g}", N) if noise else z
        c0[0, g] = O.encrypt_pk(-ish[g], s, a, e, v[g], e0, z, ps, T)[0]
    e1 = np.stack([[synth.cbd(seed, f"mk/e1{n}{g}", N) if noise else z for g in range(G)] for n in range(co)])
    e2 = np.stack([[synth.cbd(seed, f"mk/e2{n}{g}", N) if noise else z for g in range(G)] for n in range(co)])
    p1, p2 = O.masked_server_init(F, rho, b_pk, e1, e2, ps, T, lay)
    return dict(ps=ps, psis=psis, lay=lay, I=I, F=F, ip=ip, sh=sh, rho=rho, shp=shp, c0=c0, v=v, ish=ish,
                p1=p1, p2=p2)


def _identity_rhs(c):
    """Delta_Q (extract(sum_g i_g fhat_{g,n}) + sh') mod each prime, from the
    pinned packing, schoolbook product and extraction."""
    ps, lay = c["ps"], c["lay"]
    fh = O.pack_filters(c["F"], lay)
    D = O.delta_q(ps, T)
    co, G, N = fh.shape
    out = np.zeros((lay["H"], len(ps), N), np.uint32)
    for l, q in enumerate(ps):
        y = np.zeros((co, N), np.uint64)
        for n in range(co):
            for g in range(G):
                y[n] += O.negacyclic_mul(O.to_residues(c["ip"][g], q), O.to_residues(fh[n, g], q), q)
        ex = O.extract_conv((y % q).astype(np.uint64), lay)
        out[:, l, :] = ((D % q) * ((ex + np.asarray(c["shp"][0], np.uint64)) % q) % q).astype(np.uint32)
    return out


def _sum(c0r, c1r, ps):
    return np.stack([((c0r[:, l].astype(np.uint64) + c1r[:, l]) % q).astype(np.uint32)
                     for l, q in enumerate(ps)], axis=1)


def test_masked_protocol_noiseless_identity():
    c = _case(256, 2, 5, 6, 4, seed=31, noise=False)
    assert c["lay"]["G"] > 1
    c0r = O.conv_layer_masked(c["c0"], c["sh"], c["rho"], c["F"], c["shp"], c["ps"], c["psis"], T, c["lay"])[0]
    c1r = O.client_c1_masked(c["v"], c["ish"], c["p1"], c["p2"], c["ps"], c["lay"])
    np.testing.assert_array_equal(_sum(c0r, c1r, c["ps"]), _identity_rhs(c))


def test_masked_identity_needs_every_term():
    c = _case(64, 2, 3, 4, 2, seed=32, noise=False)
    rhs = _identity_rhs(c)
    ps, lay = c["ps"], c["lay"]
    c1r = O.client_c1_masked(c["v"], c["ish"], c["p1"], c["p2"], ps, lay)
    # server without its share term (as if sh were 0)
    c0_bad = O.conv_layer_masked(c["c0"], np.zeros_like(c["sh"]), c["rho"], c["F"], c["shp"], ps, c["psis"], T, lay)[0]
    assert not np.array_equal(_sum(c0_bad, c1r, ps), rhs)
    c0r = O.conv_layer_masked(c["c0"], c["sh"], c["rho"], c["F"], c["shp"], ps, c["psis"], T, lay)[0]
    # client without its mask term (v = 0), and with the mask term's sign flipped
    c1_bad = O.client_c1_masked(np.zeros_like(c["v"]), c["ish"], c["p1"], c["p2"], ps, lay)
    assert not np.array_equal(_sum(c0r, c1_bad, ps), rhs)
    c1_flip = O.client_c1_masked(-c["v"], c["ish"], c["p1"], c["p2"], ps, lay)
    assert not np.array_equal(_sum(c0r, c1_flip, ps), rhs)
    np.testing.assert_array_equal(_sum(c0r, c1r, ps), rhs)


def test_masked_protocol_with_noise_decodes_to_the_convolution():
    c = _case(256, 3, 5, 6, 4, seed=33, noise=True)
    ps, lay = c["ps"], c["lay"]
    c0r = O.conv_layer_masked(c["c0"], c["sh"], c["rho"], c["F"], c["shp"], ps, c["psis"], T, lay)[0]
    c1r = O.client_c1_masked(c["v"], c["ish"], c["p1"], c["p2"], ps, lay)
    r = _sum(c0r, c1r, ps)
    ref = O.centered(O.direct_conv(c["I"], c["F"], 1), T)
    for h in range(lay["H"]):
        m = O.centered(O.decode_scaled(r[h], ps, T) - c["shp"][0, h], T)
        for n in range(lay["co"]):
            if n // lay["s"] != h:
                continue
            for k in range(lay["h_out"]):
                for l in range(lay["w_out"]):
                    assert m[O.output_slot(lay, n, k, l)[1]] == ref[n, k, l]


def test_masked_server_tiers_agree():
    N, L, B = 512, 2, 2
    ps, psis = _params(N, L)
    lay = O.conv_layout(N, 12, 8, 4, 4)
    G, H = lay["G"], lay["H"]
    c0 = synth.residues(34, "mt/c0", (B, G, L, N), ps)
    sh = synth.ints(34, "mt/sh", (B, G, N), 0, T - 1)
    rho = synth.ints(34, "mt/rho", (8, G, N), 0, T - 1)
    shp = synth.ints(34, "mt/shp", (B, H, N), 0, T - 1)
    F = synth.ints(34, "mt/F", (8, 12, 3, 3), -128, 127)
    a = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="schoolbook")
    b = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="ntt")
    np.testing.assert_array_equal(a, b)
