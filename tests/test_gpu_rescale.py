"""he_rescale (the RNS rescale / modulus switch by the last prime) against
the oracle's definition, word for word, and through a real encryption: a
Conv layer's per-channel products rescaled from 3 to 2 limbs still decrypt
to the convolution."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu


def _gpu_rescale(p, x):
    H = U.he()
    torch = U.torch_cuda()
    cnt, L, N = x.shape
    d_out = U.empty_dev((cnt, L - 1, N))
    H.he_rescale(p, U.to_dev(x), d_out, cnt, torch.cuda.current_stream())
    H.he_sync(torch.cuda.current_stream())
    return U.from_dev(d_out).reshape(cnt, L - 1, N)


@pytest.mark.parametrize("N,L", [(8192, 3), (4096, 2), (16384, 6)])
def test_rescale_matches_oracle(N, L):
    ps, _ = U.ring(N, L)
    x = synth.residues(N + L, "rsg/x", (3, L, N), ps)
    # edge coefficients in the first polynomial: 0, Q - 1 and rounding ties
    Q = 1
    for q in ps:
        Q *= q
    qL = ps[-1]
    for k, v in enumerate([0, Q - 1, qL // 2, qL // 2 + 1, 9 * qL + qL // 2, 9 * qL + qL // 2 + 1]):
        for l, q in enumerate(ps):
            x[0, l, k] = v % q
    ref = O.rescale_last_limb(x, ps)
    with U.params(N, L) as p:
        got = _gpu_rescale(p, x)
    np.testing.assert_array_equal(got, ref)


def test_rescaled_conv_products_still_decrypt():
    H = U.he()
    N, L, ci, co, hw = 1024, 3, 5, 4, 4
    ps, psis = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    I = synth.ints(95, "rsg/I", (ci, hw, hw), -8, 7)
    F = synth.conv_weights(95, "rsg/F", co, ci, 3, 3, -128, 127)
    s = synth.ternary(95, "rsg/s", N)
    ip = O.pack_input(I, lay)
    cts = np.zeros((1, lay["G"], 2, L, N), np.uint32)
    for g in range(lay["G"]):
        cts[0, g] = O.encrypt_sk(ip[g], s, synth.residues(95, f"rsg/a{g}", (L, N), ps), synth.cbd(95, f"rsg/e{g}", N),
                                 ps, U.T)
    with U.params(N, L) as p, U.conv_bank(p, dict(ci=ci, co=co, h=hw, w=hw), F) as fb:
        y = U.run_conv(p, fb, cts, H.HE_OUT_PER_CHANNEL, co)            # [1][co][2][L][N]
        y2 = _gpu_rescale(p, y.reshape(co * 2, L, N)).reshape(co, 2, L - 1, N)
    np.testing.assert_array_equal(y2, O.rescale_last_limb(y[0], ps))
    ref = O.centered(O.direct_conv(I, F, 1), U.T)
    for n in range(co):
        m = O.decrypt(y2[n], s, ps[:-1], U.T)
        got = np.array([[m[O.output_slot(lay, n, k, l)[1]] for l in range(hw)] for k in range(hw)])
        np.testing.assert_array_equal(got, ref[n])


def test_rescale_argument_errors():
    H = U.he()
    torch = U.torch_cuda()
    with U.params(256, 1) as p:
        with pytest.raises(RuntimeError):
            H.he_rescale(p, U.to_dev(np.zeros((1, 1, 256), np.uint32)), U.empty_dev((1, 1, 256)), 1,
                         torch.cuda.current_stream())


@pytest.mark.parametrize("fin_parts", [1, 2])
def test_plan_rescales_every_output(fin_parts):
    """d_rescaled on plain and masked Conv calls of the split form, a Conv
    call of the fused form, an FC call whose window is computed directly and
    one on the transform path, in one plan: the words of the oracle's
    rescale of each call's output, on two runs in a row (the finishing
    kernel's per-polynomial counters reset themselves).  The outputs the
    finishing kernel writes are rescaled in its epilogue, the others by the
    rescale kernel; HE_PHASE_RESCALE reruns every call's rescale in that
    kernel alone.  fin_parts = 2: each output polynomial's limbs are written
    by two finishing items each, and the counters count all of them."""
    H = U.he()
    torch = U.torch_cuda()
    N, L, T = 4096, 3, U.T
    ps, psis = U.ring(N, L)
    s = torch.cuda.current_stream()
    conv = dict(ci=16, co=32, h=16, w=16)
    lay = O.conv_layout(N, 16, 32, 16, 16)
    fl = O.fc_layout(N, 64, 10)
    G, Hh, P = lay["G"], lay["H"], fl["P"]
    F = synth.conv_weights(401, "rp/F", 32, 16, 3, 3, -128, 127)
    W = synth.fc_weights(401, "rp/W", 10, 64, -128, 127)
    rho = synth.ints(401, "rp/rho", (32, G, N), 0, T - 1).astype(np.uint32)
    with U.params(N, L) as p:
        banks = [H.he_pack_filters(p, conv, F), H.he_pack_masked(p, conv, F, rho), H.he_pack_fc(p, 64, 10, W)]
        try:
            cts = U.to_dev(synth.residues(402, "rp/ct", (1, G, 2, L, N), ps))
            cts2 = U.to_dev(synth.residues(402, "rp/ct2", (2, G, 2, L, N), ps))
            c0 = U.to_dev(synth.residues(402, "rp/c0", (1, G, L, N), ps))
            sh = U.to_dev(synth.ints(402, "rp/sh", (1, G, N), 0, T - 1).astype(np.uint32))
            shp = U.to_dev(synth.ints(402, "rp/shp", (1, Hh, N), 0, T - 1).astype(np.uint32))
            fct = U.to_dev(synth.residues(402, "rp/fct", (2, 2, L, N), ps))
            fcn = U.to_dev(synth.residues(402, "rp/fcn", (2, 2, L, N), ps))
            shapes = [(1 * Hh * 2, L, N), (1 * Hh, L, N), (2 * Hh * 2, L, N), (2 * P * 2, L, N), (2 * P * 2, L, N)]
            outs = [U.empty_dev(sh_) for sh_ in shapes]
            rsc = [U.empty_dev((sh_[0], L - 1, N)) for sh_ in shapes]
            calls = [(banks[0], cts, H.HE_COEFF, outs[0], 1, None, None, rsc[0]),
                     (banks[1], c0, H.HE_COEFF, outs[1], 1, sh, shp, rsc[1]),
                     (banks[0], cts2, H.HE_COEFF, outs[2], 2, None, None, rsc[2]),
                     (banks[2], fct, H.HE_COEFF, outs[3], 2, None, None, rsc[3]),
                     (banks[2], fcn, H.HE_NTT, outs[4], 2, None, None, rsc[4])]
            # the input transforms (4096-point pairs) read their twiddles from
            # global memory with one part, from shared memory with two
            plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), fin_parts=fin_parts,
                                                      tw_smem=fin_parts - 1))
            try:
                info = H.he_plan_query(plan, len(calls))
                # split Conv (scalar MAC), fused-form Conv, direct FC, FC on the transform path
                assert info["form"] == [1, 1, 0, 3, 0]
                assert info["rescale_fused_calls"] == 3          # calls 0, 1 and 4
                assert info["rescale_items"] > 0                 # calls 2 and 3
                for run in range(2):
                    for r in rsc:
                        r.fill_(-1)
                    H.he_plan_run(plan, s)
                    H.he_sync(s)
                    H.he_plan_check(plan)
                    for o, r, sh_ in zip(outs, rsc, shapes):
                        want = O.rescale_last_limb(U.from_dev(o).reshape(sh_), ps)
                        np.testing.assert_array_equal(U.from_dev(r).reshape(want.shape), want)
                for r in rsc:
                    r.fill_(-1)
                H.he_plan_run_phase(plan, H.HE_PHASE_RESCALE, s)
                H.he_sync(s)
                for o, r, sh_ in zip(outs, rsc, shapes):
                    want = O.rescale_last_limb(U.from_dev(o).reshape(sh_), ps)
                    np.testing.assert_array_equal(U.from_dev(r).reshape(want.shape), want)
            finally:
                H.he_plan_destroy(plan)
            with U.params(N, 1) as p1:
                f1 = H.he_pack_filters(p1, conv, F)
                try:
                    x1 = U.to_dev(np.zeros((1, G, 2, 1, N), np.uint32))
                    with pytest.raises(RuntimeError):   # one limb: nothing to rescale by
                        H.he_plan_create([(f1, x1, H.HE_COEFF, U.empty_dev((1, Hh, 2, 1, N)), 1, None, None,
                                           U.empty_dev((Hh * 2, 1, N)))])
                finally:
                    H.he_filters_destroy(f1)
        finally:
            for b in banks:
                H.he_filters_destroy(b)
