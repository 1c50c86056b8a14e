"""The paper's masked server step (Alg. 1) on the GPU: he_pack_masked +
he_conv_layer_masked against the oracle's conv_layer_masked, word for word,
and the whole protocol (GPU server step, oracle client) decoding to the
plaintext convolution."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu

T = U.T


def _masked_case(N, L, ci, co, hw, B, seed):
    ps, psis = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    G, H = lay["G"], lay["H"]
    c0 = synth.residues(seed, "gm/c0", (B, G, L, N), ps)
    sh = synth.ints(seed, "gm/sh", (B, G, N), 0, T - 1).astype(np.uint32)
    rho = synth.ints(seed, "gm/rho", (co, G, N), 0, T - 1).astype(np.uint32)
    shp = synth.ints(seed, "gm/shp", (B, H, N), 0, T - 1).astype(np.uint32)
    F = synth.conv_weights(seed, "gm/F", co, ci, 3, 3, -128, 127)
    return ps, psis, lay, c0, sh, rho, shp, F


def _run_masked(p, f, c0, sh, shp, dom, B, H):
    H_ = U.he()
    torch = U.torch_cuda()
    _, _, L, N = c0.shape
    U.reserve(p, 2 * c0.size * 4)  # c0 and sh transformed side by side
    d_out = U.empty_dev((B, H, L, N))
    H_.he_conv_layer_masked(p, f, U.to_dev(c0), U.to_dev(sh), U.to_dev(shp), dom, d_out, B,
                            torch.cuda.current_stream())
    H_.he_sync(torch.cuda.current_stream())
    return U.from_dev(d_out).reshape(B, H, L, N)


# (N, L, ci, co, hw, B, in_domain): G = 1 and G > 1, odd B (one column per CTA), 3 limbs
CASES = [(256, 2, 5, 6, 4, 1, "coeff"), (512, 2, 12, 8, 4, 2, "ntt"), (1024, 3, 16, 16, 8, 3, "coeff"),
         (2048, 1, 3, 4, 16, 1, "ntt")]


@pytest.mark.parametrize("N,L,ci,co,hw,B,dom", CASES)
def test_masked_server_step_matches_oracle(N, L, ci, co, hw, B, dom):
    H = U.he()
    ps, psis, lay, c0, sh, rho, shp, F = _masked_case(N, L, ci, co, hw, B, seed=N + ci + B)
    ref = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="ntt")
    x = c0
    if dom == "ntt":
        x = c0.copy()
        for l in range(L):
            x[:, :, l, :] = O.ntt_fwd(np.ascontiguousarray(c0[:, :, l, :]), ps[l], psis[l])
    with U.params(N, L) as p:
        f = H.he_pack_masked(p, dict(ci=ci, co=co, h=hw, w=hw), F, rho)
        try:
            for _ in range(2):  # repeatable
                got = _run_masked(p, f, x, sh, shp, H.HE_NTT if dom == "ntt" else H.HE_COEFF, B, lay["H"])
                np.testing.assert_array_equal(got, ref)
        finally:
            H.he_filters_destroy(f)


def test_masked_plain20_shape_full_size():
    """A plain-20 layer shape (16 -> 32 at 32x32, N = 8192, 3 limbs): every
    word against the oracle's NTT tier."""
    H = U.he()
    N, L, B = 8192, 3, 1
    ps, psis, lay, c0, sh, rho, shp, F = _masked_case(N, L, 16, 32, 32, B, seed=61)
    ref = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_masked(p, dict(ci=16, co=32, h=32, w=32), F, rho)
        try:
            got = _run_masked(p, f, c0, sh, shp, H.HE_COEFF, B, lay["H"])
        finally:
            H.he_filters_destroy(f)
    np.testing.assert_array_equal(got, ref)


def test_masked_protocol_on_gpu_decodes_to_the_convolution():
    """Alg. 1 end to end: the client encrypts -(i + sh) (c0 only), the GPU
    evaluates the masked server step, the client adds its c1 share computed
    from p1 / p2 and decodes without the secret key: the result minus sh' is
    the plaintext convolution mod t at every valid slot."""
    H = U.he()
    N, L, ci, co, hw, seed = 256, 3, 5, 6, 4, 71
    ps, psis = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    G, Hh = lay["G"], lay["H"]
    I = synth.ints(seed, "gp/I", (ci, hw, hw), -8, 7)
    F = synth.conv_weights(seed, "gp/F", co, ci, 3, 3, -128, 127)
    ip = O.pack_input(I, lay)
    sh = synth.ints(seed, "gp/sh", (1, G, N), 0, T - 1)
    rho = synth.ints(seed, "gp/rho", (co, G, N), 0, T - 1)
    shp = synth.ints(seed, "gp/shp", (1, Hh, N), 0, T - 1)
    s = synth.ternary(seed, "gp/s", N)
    a = synth.residues(seed, "gp/a", (L, N), ps)
    e = synth.cbd(seed, "gp/e", N)
    b_pk = np.zeros((L, N), np.uint32)
    for l, q in enumerate(ps):
        b_pk[l] = ((-O.negacyclic_mul(a[l], O.to_residues(s, q), q).astype(np.int64) + e) % q).astype(np.uint32)
    ish = ip + sh[0]
    c0 = np.zeros((1, G, L, N), np.uint32)
    v = np.zeros((G, N), np.int64)
    z = np.zeros(N, np.int64)
    for g in range(G):
        v[g] = synth.v_poly(seed, f"gp/v{g}", N)
        c0[0, g] = O.encrypt_pk(-ish[g], s, a, e, v[g], synth.cbd(seed, f"gp/e0{g}", N), z, ps, T)[0]
    e1 = np.stack([[synth.cbd(seed, f"gp/e1{n}{g}", N) for g in range(G)] for n in range(co)])
    e2 = np.stack([[synth.cbd(seed, f"gp/e2{n}{g}", N) for g in range(G)] for n in range(co)])
    p1, p2 = O.masked_server_init(F, rho, b_pk, e1, e2, ps, T, lay)
    with U.params(N, L) as p:
        f = H.he_pack_masked(p, dict(ci=ci, co=co, h=hw, w=hw), F, rho.astype(np.uint32))
        try:
            c0r = _run_masked(p, f, c0, sh.astype(np.uint32), shp.astype(np.uint32), H.HE_COEFF, 1, Hh)[0]
        finally:
            H.he_filters_destroy(f)
    c1r = O.client_c1_masked(v, ish, p1, p2, ps, lay)
    r = np.stack([((c0r[:, l].astype(np.uint64) + c1r[:, l]) % q).astype(np.uint32) for l, q in enumerate(ps)], 1)
    ref = O.centered(O.direct_conv(I, F, 1), T)
    for h in range(Hh):
        m = O.centered(O.decode_scaled(r[h], ps, T) - shp[0, h], T)
        for n in range(co):
            if n // lay["s"] != h:
                continue
            for k in range(lay["h_out"]):
                for l in range(lay["w_out"]):
                    assert m[O.output_slot(lay, n, k, l)[1]] == ref[n, k, l]


def test_masked_argument_errors():
    H = U.he()
    torch = U.torch_cuda()
    N, L, ci, co, hw = 256, 2, 5, 6, 4
    ps, psis, lay, c0, sh, rho, shp, F = _masked_case(N, L, ci, co, hw, 1, seed=81)
    desc = dict(ci=ci, co=co, h=hw, w=hw)
    with U.params(N, L) as p:
        bad = rho.copy()
        bad[0, 0, 3] = T
        with pytest.raises(RuntimeError):
            H.he_pack_masked(p, desc, F, bad)
        fm = H.he_pack_masked(p, desc, F, rho)
        fr = H.he_pack_filters(p, desc, F)
        try:
            d_in = U.to_dev(np.zeros((1, lay["G"], 2, L, N), np.uint32))
            d_out = U.empty_dev((1, lay["H"], 2, L, N))
            with pytest.raises(RuntimeError):   # a masked bank in the ordinary call
                H.he_conv_layer(p, fm, d_in, H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, 1, torch.cuda.current_stream())
            with pytest.raises(RuntimeError):   # an ordinary bank in the masked call
                H.he_conv_layer_masked(p, fr, U.to_dev(c0), U.to_dev(sh), U.to_dev(shp), H.HE_COEFF,
                                       U.empty_dev((1, lay["H"], L, N)), 1, torch.cuda.current_stream())
            with pytest.raises(RuntimeError):   # masked banks do not run in plans
                H.he_plan_create([(fm, d_in, H.HE_COEFF, d_out, 1)])
        finally:
            H.he_filters_destroy(fm)
            H.he_filters_destroy(fr)


def _protocol_case(N, L, ci, co, hw, seed):
    ps, psis = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    G, Hh = lay["G"], lay["H"]
    I = synth.ints(seed, "cp/I", (ci, hw, hw), -8, 7)
    F = synth.conv_weights(seed, "cp/F", co, ci, 3, 3, -128, 127)
    ip = O.pack_input(I, lay)
    sh = synth.ints(seed, "cp/sh", (1, G, N), 0, T - 1)
    rho = synth.ints(seed, "cp/rho", (co, G, N), 0, T - 1)
    shp = synth.ints(seed, "cp/shp", (1, Hh, N), 0, T - 1)
    s = synth.ternary(seed, "cp/s", N)
    a = synth.residues(seed, "cp/a", (L, N), ps)
    e = synth.cbd(seed, "cp/e", N)
    b_pk = np.zeros((L, N), np.uint32)
    for l, q in enumerate(ps):
        b_pk[l] = ((-O.negacyclic_mul(a[l], O.to_residues(s, q), q).astype(np.int64) + e) % q).astype(np.uint32)
    ish = ip + sh[0]
    c0 = np.zeros((1, G, L, N), np.uint32)
    v = np.zeros((G, N), np.int64)
    z = np.zeros(N, np.int64)
    for g in range(G):
        v[g] = synth.v_poly(seed, f"cp/v{g}", N)
        c0[0, g] = O.encrypt_pk(-ish[g], s, a, e, v[g], synth.cbd(seed, f"cp/e0{g}", N), z, ps, T)[0]
    e1 = np.stack([[synth.cbd(seed, f"cp/e1{n}{g}", N) for g in range(G)] for n in range(co)])
    e2 = np.stack([[synth.cbd(seed, f"cp/e2{n}{g}", N) for g in range(G)] for n in range(co)])
    p1, p2 = O.masked_server_init(F, rho, b_pk, e1, e2, ps, T, lay)
    return dict(ps=ps, psis=psis, lay=lay, I=I, F=F, sh=sh, rho=rho, shp=shp, c0=c0, v=v, ish=ish, p1=p1, p2=p2)


def _run_client(p, f, v, ish, B, Hh, L, N):
    H = U.he()
    torch = U.torch_cuda()
    U.reserve(p, 2 * np.asarray(v).size * L * 4)  # -v and i + sh in every limb
    d_out = U.empty_dev((B, Hh, L, N))
    H.he_conv_client(p, f, torch.from_numpy(np.ascontiguousarray(v, np.int32).ravel()).cuda(),
                     torch.from_numpy(np.ascontiguousarray(ish, np.int32).ravel()).cuda(), d_out, B,
                     torch.cuda.current_stream())
    H.he_sync(torch.cuda.current_stream())
    return U.from_dev(d_out).reshape(B, Hh, L, N)


def test_client_step_matches_oracle():
    H = U.he()
    c = _protocol_case(512, 2, 12, 8, 4, seed=91)
    lay, ps = c["lay"], c["ps"]
    N, L = lay["N"], len(ps)
    ref = O.client_c1_masked(c["v"], c["ish"], c["p1"], c["p2"], ps, lay)
    with U.params(N, L) as p:
        f = H.he_pack_client(p, dict(ci=12, co=8, h=4, w=4), c["p1"], c["p2"])
        try:
            got = _run_client(p, f, c["v"][None], c["ish"][None], 1, lay["H"], L, N)[0]
        finally:
            H.he_filters_destroy(f)
    np.testing.assert_array_equal(got, ref)


def test_whole_protocol_on_gpu_decodes_to_the_convolution():
    """Server step and client step both on the GPU (he_conv_layer_masked,
    he_conv_client); the oracle only encrypts, prepares p1 / p2 and decodes."""
    H = U.he()
    ci, co, hw = 5, 6, 4
    c = _protocol_case(256, 3, ci, co, hw, seed=92)
    lay, ps = c["lay"], c["ps"]
    N, L, Hh = lay["N"], len(ps), lay["H"]
    desc = dict(ci=ci, co=co, h=hw, w=hw)
    with U.params(N, L) as p:
        fs = H.he_pack_masked(p, desc, c["F"], c["rho"].astype(np.uint32))
        fc = H.he_pack_client(p, desc, c["p1"], c["p2"])
        try:
            c0r = _run_masked(p, fs, c["c0"], c["sh"].astype(np.uint32), c["shp"].astype(np.uint32), H.HE_COEFF, 1, Hh)[0]
            c1r = _run_client(p, fc, c["v"][None], c["ish"][None], 1, Hh, L, N)[0]
        finally:
            H.he_filters_destroy(fs)
            H.he_filters_destroy(fc)
    r = np.stack([((c0r[:, l].astype(np.uint64) + c1r[:, l]) % q).astype(np.uint32) for l, q in enumerate(ps)], 1)
    ref = O.centered(O.direct_conv(c["I"], c["F"], 1), T)
    for h in range(Hh):
        m = O.centered(O.decode_scaled(r[h], ps, T) - c["shp"][0, h], T)
        for n in range(co):
            if n // lay["s"] != h:
                continue
            for k in range(lay["h_out"]):
                for l in range(lay["w_out"]):
                    assert m[O.output_slot(lay, n, k, l)[1]] == ref[n, k, l]
