"""The masked FC step of Alg. 2 on the GPU: he_pack_fc_masked +
he_fc_layer_masked (server) and he_pack_fc_client + he_fc_client (client)
against the oracle word for word, and the whole protocol with both steps on
the GPU decoding to W I + B."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu

T = U.T


def _ntt(x, ps, psis):
    x = x.copy()
    for l in range(len(ps)):
        x[..., l, :] = O.ntt_fwd(np.ascontiguousarray(x[..., l, :]), ps[l], psis[l])
    return x


def _server(p, f, c0, sh, shp, dom, B, P):
    H = U.he()
    torch = U.torch_cuda()
    _, L, N = c0.shape
    U.reserve(p, U.he().he_fc_workspace_bytes(p, B))
    d_out = U.empty_dev((B, P, L, N))
    H.he_fc_layer_masked(p, f, U.to_dev(c0), U.to_dev(sh), U.to_dev(shp), dom, d_out, B,
                         torch.cuda.current_stream())
    H.he_sync(torch.cuda.current_stream())
    return U.from_dev(d_out).reshape(B, P, L, N)


def _client(p, f, v, ish, B, P, L, N):
    H = U.he()
    torch = U.torch_cuda()
    U.reserve(p, H.he_fc_workspace_bytes(p, B))
    d_out = U.empty_dev((B, P, L, N))
    H.he_fc_client(p, f, torch.from_numpy(np.ascontiguousarray(v, np.int32).ravel()).cuda(),
                   torch.from_numpy(np.ascontiguousarray(ish, np.int32).ravel()).cuda(), d_out, B,
                   torch.cuda.current_stream())
    H.he_sync(torch.cuda.current_stream())
    return U.from_dev(d_out).reshape(B, P, L, N)


# (N, L, n_in, n_out, B, in_domain, bias): P = 1 and P > 1 with a ragged last
# block, odd B, NTT-domain c0, plain-20's FC (64 -> 10) and the wide x4
# network's (256 -> 100) at full size
CASES = [(256, 2, 20, 12, 1, "coeff", True), (1024, 3, 100, 40, 3, "ntt", False),
         (8192, 3, 64, 10, 1, "coeff", True), (16384, 6, 256, 100, 2, "coeff", True)]


@pytest.mark.parametrize("N,L,n_in,n_out,B,dom,bias", CASES)
def test_masked_fc_server_step_matches_oracle(N, L, n_in, n_out, B, dom, bias):
    H = U.he()
    ps, psis = U.ring(N, L)
    lay = O.fc_layout(N, n_in, n_out)
    P = lay["P"]
    seed = N + n_in + B
    c0 = synth.residues(seed, "gf/c0", (B, L, N), ps)
    sh = synth.ints(seed, "gf/sh", (B, N), 0, T - 1).astype(np.uint32)
    rho = synth.ints(seed, "gf/rho", (P, N), 0, T - 1).astype(np.uint32)
    shp = synth.ints(seed, "gf/shp", (B, P, N), 0, T - 1).astype(np.uint32)
    W = synth.fc_weights(seed, "gf/W", n_out, n_in, -128, 127)
    Bv = synth.ints(seed, "gf/B", (n_out,), -3000, 3000).astype(np.int32) if bias else None
    ref = O.fc_layer_masked(c0, sh, rho, W, Bv, shp, ps, psis, T, lay, tier="ntt")
    x = _ntt(c0, ps, psis) if dom == "ntt" else c0
    with U.params(N, L) as p:
        f = H.he_pack_fc_masked(p, n_in, n_out, W, Bv, rho)
        try:
            for _ in range(2):  # repeatable: every word rewritten
                got = _server(p, f, x, sh, shp, H.HE_NTT if dom == "ntt" else H.HE_COEFF, B, P)
                np.testing.assert_array_equal(got, ref)
        finally:
            H.he_filters_destroy(f)


def _protocol(N, L, n_in, n_out, seed):
    ps, psis = U.ring(N, L)
    lay = O.fc_layout(N, n_in, n_out)
    P = lay["P"]
    I = synth.ints(seed, "fp/I", (n_in,), -8, 7)
    W = synth.fc_weights(seed, "fp/W", n_out, n_in, -128, 127)
    Bv = synth.ints(seed, "fp/B", (n_out,), -500, 500).astype(np.int32)
    sh = synth.ints(seed, "fp/sh", (1, N), 0, T - 1)
    rho = synth.ints(seed, "fp/rho", (P, N), 0, T - 1)
    shp = synth.ints(seed, "fp/shp", (1, P, N), 0, T - 1)
    s = synth.ternary(seed, "fp/s", N)
    a = synth.residues(seed, "fp/a", (L, N), ps)
    e = synth.cbd(seed, "fp/e", N)
    b_pk = np.zeros((L, N), np.uint32)
    for l, q in enumerate(ps):
        b_pk[l] = ((-O.negacyclic_mul(a[l], O.to_residues(s, q), q).astype(np.int64) + e) % q).astype(np.uint32)
    ish = O.pack_fc_input(I, lay) + sh[0]
    v = synth.v_poly(seed, "fp/v", N)
    z = np.zeros(N, np.int64)
    c0 = O.encrypt_pk(-ish, s, a, e, v, synth.cbd(seed, "fp/e0", N), z, ps, T)[0][None]
    e1 = np.stack([synth.cbd(seed, f"fp/e1{j}", N) for j in range(P)])
    e2 = np.stack([synth.cbd(seed, f"fp/e2{j}", N) for j in range(P)])
    p1, p2 = O.masked_fc_server_init(W, rho, b_pk, e1, e2, ps, T, lay)
    return dict(ps=ps, psis=psis, lay=lay, I=I, W=W, Bv=Bv, sh=sh, rho=rho, shp=shp, c0=c0, v=v, ish=ish,
                p1=p1, p2=p2)


def test_masked_fc_client_step_matches_oracle():
    H = U.he()
    c = _protocol(1024, 2, 100, 40, seed=93)
    lay, ps = c["lay"], c["ps"]
    N, L, P = lay["N"], len(ps), lay["P"]
    assert P > 1
    ref = O.client_c1_fc_masked(c["v"], c["ish"], c["p1"], c["p2"], ps, lay)
    with U.params(N, L) as p:
        f = H.he_pack_fc_client(p, 100, 40, c["p1"], c["p2"])
        try:
            got = _client(p, f, c["v"][None], c["ish"][None], 1, P, L, N)[0]
        finally:
            H.he_filters_destroy(f)
    np.testing.assert_array_equal(got, ref)


def test_whole_masked_fc_protocol_on_gpu_decodes_to_w_i_plus_b():
    """Server and client steps on the GPU; the oracle only encrypts, prepares
    p1 / p2 and decodes without the secret key."""
    H = U.he()
    n_in, n_out = 64, 10
    c = _protocol(512, 3, n_in, n_out, seed=94)
    lay, ps = c["lay"], c["ps"]
    N, L, P = lay["N"], len(ps), lay["P"]
    with U.params(N, L) as p:
        fs = H.he_pack_fc_masked(p, n_in, n_out, c["W"], c["Bv"], c["rho"].astype(np.uint32))
        fc = H.he_pack_fc_client(p, n_in, n_out, c["p1"], c["p2"])
        try:
            c0r = _server(p, fs, c["c0"], c["sh"].astype(np.uint32), c["shp"].astype(np.uint32), H.HE_COEFF, 1, P)[0]
            c1r = _client(p, fc, c["v"][None], c["ish"][None], 1, P, L, N)[0]
        finally:
            H.he_filters_destroy(fs)
            H.he_filters_destroy(fc)
    r = np.stack([((c0r[:, l].astype(np.uint64) + c1r[:, l]) % q).astype(np.uint32) for l, q in enumerate(ps)], 1)
    want = O.centered(O.direct_fc(c["W"], c["I"], c["Bv"]), T)
    rr = lay["rows_per_poly"]
    for j in range(P):
        m = O.centered(O.decode_scaled(r[j], ps, T) - c["shp"][0, j], T)
        np.testing.assert_array_equal(m[:lay["rows"][j]], want[j * rr: j * rr + lay["rows"][j]])


def test_masked_fc_argument_errors():
    H = U.he()
    torch = U.torch_cuda()
    N, L, n_in, n_out = 256, 2, 20, 12
    lay = O.fc_layout(N, n_in, n_out)
    P = lay["P"]
    W = synth.fc_weights(5, "fe/W", n_out, n_in, -128, 127)
    rho = synth.ints(5, "fe/rho", (P, N), 0, T - 1).astype(np.uint32)
    with U.params(N, L) as p:
        bad = rho.copy()
        bad[1, 7] = T
        with pytest.raises(RuntimeError):
            H.he_pack_fc_masked(p, n_in, n_out, W, None, bad)
        fm = H.he_pack_fc_masked(p, n_in, n_out, W, None, rho)
        fo = H.he_pack_fc(p, n_in, n_out, W)
        try:
            s = torch.cuda.current_stream()
            d_in = U.to_dev(np.zeros((1, 2, L, N), np.uint32))
            d_out = U.empty_dev((1, P, 2, L, N))
            c0, sh, shp = U.to_dev(np.zeros((1, L, N), np.uint32)), U.to_dev(np.zeros((1, N), np.uint32)), \
                U.to_dev(np.zeros((1, P, N), np.uint32))
            with pytest.raises(RuntimeError):   # a masked bank in the ordinary FC call
                H.he_fc_layer(p, fm, d_in, H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, 1, s)
            with pytest.raises(RuntimeError):   # an ordinary bank in the masked call
                H.he_fc_layer_masked(p, fo, c0, sh, shp, H.HE_COEFF, U.empty_dev((1, P, L, N)), 1, s)
            with pytest.raises(RuntimeError):   # a server bank in the client call
                zi = torch.zeros(N, dtype=torch.int32, device="cuda")
                H.he_fc_client(p, fm, zi, zi, U.empty_dev((1, P, L, N)), 1, s)
            with pytest.raises(RuntimeError):   # masked banks do not run in plans
                H.he_plan_create([(fm, d_in, H.HE_COEFF, d_out, 1)])
        finally:
            H.he_filters_destroy(fm)
            H.he_filters_destroy(fo)
