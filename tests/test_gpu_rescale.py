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
