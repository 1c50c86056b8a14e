"""Other layer families (5x5 filters of the f5 variant, the 3x3 layers of
the w3 variants at 48 / 96 / 192 channels, ResNet-style 1x1 layers with
c_o < c_i and c_o > c_i, and their 3x3 layers at 14x14) at full size,
N = 8192 and 3 limbs: a plan, single calls and the oracle give the same
words (every word of every limb by the oracle's NTT tier, and sampled words
by its schoolbook dot products, an independent tier).  Every layer with an interleave
s >= 4 takes the split form in the plan, its input groups taken in parts of
8, 4, 2 or 1 (G = 12, 6, 3, 32 have 3, 3, 3, 4 parts)."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu

# (ci, co, hw, f, pad, N, L)
SHAPES = [(48, 48, 32, 5, 2, 8192, 3), (96, 192, 16, 5, 2, 8192, 3), (192, 192, 8, 5, 2, 8192, 3),
          (3, 48, 32, 5, 2, 8192, 3), (1024, 256, 14, 1, 0, 8192, 3), (256, 1024, 14, 1, 0, 8192, 3),
          (256, 256, 14, 3, 1, 8192, 3), (64, 64, 32, 3, 1, 16384, 2),
          (3, 48, 32, 3, 1, 8192, 3), (48, 48, 32, 3, 1, 8192, 3), (48, 96, 32, 3, 1, 8192, 3),
          (96, 96, 16, 3, 1, 8192, 3), (96, 192, 16, 3, 1, 8192, 3), (192, 192, 8, 3, 1, 8192, 3)]


@pytest.mark.parametrize("ci,co,hw,f,pad,N,L", SHAPES)
def test_layer_family_full_size(ci, co, hw, f, pad, N, L):
    H = U.he()
    torch = U.torch_cuda()
    B = 1
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=ci + co + f, fh=f, fw=f, pad=pad)
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as fb:
        single = U.run_conv(p, fb, cts, H.HE_OUT_EXTRACTED, lay["H"])
        d_in = U.to_dev(cts)
        # finishing items over all residue classes, and over quarters of them
        for fin_parts in (1, 4):
            d_out = U.empty_dev(single.shape)
            plan = H.he_plan_create_tuned([(fb, d_in, H.HE_COEFF, d_out, B)],
                                          dict(H.he_plan_tuning_default(), fin_parts=fin_parts))
            # s >= 4: the split form, groups in parts (G = 8: the larger input buffers)
            if lay["s"] >= 4:
                assert H.he_plan_query(plan, 1)["form"][0] == 1
            try:
                H.he_plan_run(plan, torch.cuda.current_stream())
                H.he_sync(torch.cuda.current_stream())
                H.he_plan_check(plan)
            finally:
                H.he_plan_destroy(plan)
            got = U.from_dev(d_out).reshape(single.shape)
            np.testing.assert_array_equal(got, single, err_msg=f"fin_parts {fin_parts}")
    ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
    np.testing.assert_array_equal(got, ref)
    rng = np.random.default_rng(co)
    picks = [(0, int(rng.integers(lay["H"])), int(rng.integers(2)), int(rng.integers(L)), int(rng.integers(N)))
             for _ in range(16)]
    np.testing.assert_array_equal(O.conv_layer_sampled(cts, F, ps, lay, picks),
                                  np.array([got[pk] for pk in picks], dtype=np.uint32))


def test_f5_workload_decrypts_to_the_convolution():
    """One 5x5 layer through real RLWE: secret-key encryption of a packed
    image, the GPU layer in per-channel mode, decryption equals the direct
    convolution mod t at every output position (N = 4096, 3 limbs)."""
    H = U.he()
    N, L, ci, co, hw = 4096, 3, 6, 4, 8
    ps, psis = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw, 5, 5, 2)
    I = synth.ints(91, "f5/I", (ci, hw, hw), -8, 7)
    F = synth.conv_weights(91, "f5/F", co, ci, 5, 5, -128, 127)
    s = synth.ternary(91, "f5/s", N)
    ip = O.pack_input(I, lay)
    cts = np.zeros((1, lay["G"], 2, L, N), np.uint32)
    for g in range(lay["G"]):
        a = synth.residues(91, f"f5/a{g}", (L, N), ps)
        cts[0, g] = O.encrypt_sk(ip[g], s, a, synth.cbd(91, f"f5/e{g}", N), ps, U.T)
    with U.params(N, L) as p, U.conv_bank(p, dict(ci=ci, co=co, h=hw, w=hw, fh=5, fw=5, pad=2), F) as fb:
        y = U.run_conv(p, fb, cts, H.HE_OUT_PER_CHANNEL, co)
    ref = O.centered(O.direct_conv(I, F, 2), U.T)
    for n in range(co):
        m = O.decrypt(y[0, n], s, ps, U.T)
        got = np.array([[m[O.output_slot(lay, n, k, l)[1]] for l in range(lay["w_out"])] for k in range(lay["h_out"])])
        np.testing.assert_array_equal(got, ref[n])
