"""Pins for the oracle's masked FC protocol (Alg. 2): the server step, the
client's share and the key-free decode.

* Noiseless identity: with every error polynomial 0, c0^r + c1^r equals
  Delta_Q ((W I + B)_{j r + k} + sh'_j[k]) at the window coefficients
  k < rows_j of block j and Delta_Q sh'_j[k] elsewhere, modulo every prime.
  The right-hand side is the plain matrix-vector product: nothing of the
  packing enters it.
* The identity fails when the server drops its share term, when the client
  drops its mask term or flips its sign, and when the bias is left out.
* With RLWE noise the decode minus sh' is W I + B in every window.
* The schoolbook and NTT tiers of the masked FC server step agree.
"""

import numpy as np

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537


def _case(N, L, n_in, n_out, seed, noise, bias=True):
    ps = O.select_primes(N, L)
    psis = [O.root_2n(q, N) for q in ps]
    lay = O.fc_layout(N, n_in, n_out)
    P = lay["P"]
    I = synth.ints(seed, "mf/I", (n_in,), -8, 7)
    W = synth.ints(seed, "mf/W", (n_out, n_in), -128, 127)
    Bv = synth.ints(seed, "mf/B", (n_out,), -500, 500) if bias else None
    ip = O.pack_fc_input(I, lay)
    sh = synth.ints(seed, "mf/sh", (1, N), 0, T - 1)
    rho = synth.ints(seed, "mf/rho", (P, N), 0, T - 1)
    shp = synth.ints(seed, "mf/shp", (1, P, N), 0, T - 1)
    s = synth.ternary(seed, "mf/s", N)
    a = synth.residues(seed, "mf/a", (L, N), ps)
    z = np.zeros(N, np.int64)
    e = synth.cbd(seed, "mf/e", N) if noise else z
    b_pk = np.zeros((L, N), np.uint32)
    for l, q in enumerate(ps):
        b_pk[l] = ((-O.negacyclic_mul(a[l], O.to_residues(s, q), q).astype(np.int64) + e) % q).astype(np.uint32)
    ish = ip + sh[0]
    v = synth.v_poly(seed, "mf/v", N)
    e0 = synth.cbd(seed, "mf/e0", N) if noise else z
    c0 = O.encrypt_pk(-ish, s, a, e, v, e0, z, ps, T)[0][None]          # [1][L][N]
    e1 = np.stack([synth.cbd(seed, f"mf/e1{j}", N) if noise else z for j in range(P)])
    e2 = np.stack([synth.cbd(seed, f"mf/e2{j}", N) if noise else z for j in range(P)])
    p1, p2 = O.masked_fc_server_init(W, rho, b_pk, e1, e2, ps, T, lay)
    return dict(ps=ps, psis=psis, lay=lay, I=I, W=W, Bv=Bv, sh=sh, rho=rho, shp=shp, c0=c0, v=v, ish=ish,
                p1=p1, p2=p2)


def _server(c, **kw):
    args = dict(c0=c["c0"], sh=c["sh"], rho=c["rho"], W=c["W"], Bv=c["Bv"], shp=c["shp"])
    args.update(kw)
    return O.fc_layer_masked(args["c0"], args["sh"], args["rho"], args["W"], args["Bv"], args["shp"],
                             c["ps"], c["psis"], T, c["lay"])[0]


def _client(c, v=None):
    return O.client_c1_fc_masked(c["v"] if v is None else v, c["ish"], c["p1"], c["p2"], c["ps"], c["lay"])


def _identity_rhs(c):
    """Delta_Q (W I + B + sh') on each window, Delta_Q sh' elsewhere."""
    ps, lay = c["ps"], c["lay"]
    Bv = c["Bv"] if c["Bv"] is not None else np.zeros(lay["n_out"], np.int64)
    y = np.asarray(c["W"], np.int64) @ np.asarray(c["I"], np.int64) + np.asarray(Bv, np.int64)
    D = O.delta_q(ps, T)
    P, N, r = lay["P"], lay["N"], lay["rows_per_poly"]
    m = np.asarray(c["shp"][0], np.int64).copy()                          # [P][N]
    for j in range(P):
        m[j, :lay["rows"][j]] += y[j * r: j * r + lay["rows"][j]]
    out = np.zeros((P, len(ps), N), np.uint32)
    for l, q in enumerate(ps):
        out[:, l, :] = [[(D % q) * (int(x) % q) % q for x in row] for row in m]
    return out


def _sum(a, b, ps):
    return np.stack([((a[:, l].astype(np.uint64) + b[:, l]) % q).astype(np.uint32) for l, q in enumerate(ps)], axis=1)


def test_masked_fc_noiseless_identity_is_the_matrix_vector_product():
    c = _case(256, 2, 20, 12, seed=41, noise=False)
    assert c["lay"]["P"] == 2 and c["lay"]["rows"] == [8, 4]
    np.testing.assert_array_equal(_sum(_server(c), _client(c), c["ps"]), _identity_rhs(c))


def test_masked_fc_identity_needs_every_term():
    c = _case(128, 2, 16, 10, seed=42, noise=False)
    rhs = _identity_rhs(c)
    c1 = _client(c)
    assert not np.array_equal(_sum(_server(c, sh=np.zeros_like(c["sh"])), c1, c["ps"]), rhs)
    assert not np.array_equal(_sum(_server(c, Bv=None), c1, c["ps"]), rhs)
    c0r = _server(c)
    assert not np.array_equal(_sum(c0r, _client(c, v=np.zeros_like(c["v"])), c["ps"]), rhs)
    assert not np.array_equal(_sum(c0r, _client(c, v=-c["v"]), c["ps"]), rhs)
    np.testing.assert_array_equal(_sum(c0r, c1, c["ps"]), rhs)


def test_masked_fc_with_noise_decodes_to_w_i_plus_b():
    c = _case(512, 3, 64, 10, seed=43, noise=True)
    ps, lay = c["ps"], c["lay"]
    r = _sum(_server(c), _client(c), ps)
    want = O.centered(O.direct_fc(c["W"], c["I"], c["Bv"]), T)
    rr = lay["rows_per_poly"]
    for j in range(lay["P"]):
        m = O.centered(O.decode_scaled(r[j], ps, T) - c["shp"][0, j], T)
        np.testing.assert_array_equal(m[:lay["rows"][j]], want[j * rr: j * rr + lay["rows"][j]])


def test_masked_fc_tiers_agree():
    N, L, B = 512, 2, 3
    ps = O.select_primes(N, L)
    psis = [O.root_2n(q, N) for q in ps]
    lay = O.fc_layout(N, 100, 20)
    P = lay["P"]
    c0 = synth.residues(44, "mft/c0", (B, L, N), ps)
    sh = synth.ints(44, "mft/sh", (B, N), 0, T - 1)
    rho = synth.ints(44, "mft/rho", (P, N), 0, T - 1)
    shp = synth.ints(44, "mft/shp", (B, P, N), 0, T - 1)
    W = synth.ints(44, "mft/W", (20, 100), -128, 127)
    Bv = synth.ints(44, "mft/B", (20,), -100, 100)
    a = O.fc_layer_masked(c0, sh, rho, W, Bv, shp, ps, psis, T, lay, tier="schoolbook")
    b = O.fc_layer_masked(c0, sh, rho, W, Bv, shp, ps, psis, T, lay, tier="ntt")
    np.testing.assert_array_equal(a, b)
