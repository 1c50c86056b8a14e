"""The tensor-core channel MAC (banks packed with he_pack_filters_for_batch):
plan calls of 1 to 8 ciphertexts on it must give exactly the oracle's words,
and the same words as the scalar kernels on the ordinary bank.  Single calls
and plan calls of more than 8 ciphertexts read the same bank through the
scalar kernels."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu


def _ntt_inputs(x, ps, psis):
    x = x.copy()
    for l in range(len(ps)):
        x[..., l, :] = O.ntt_fwd(np.ascontiguousarray(x[..., l, :]), ps[l], psis[l])
    return x


def test_tensor_core_layout_is_chosen_by_batch_and_shape():
    H = U.he()
    N, L = 4096, 2
    with U.params(N, L) as p:
        for (ci, co, hw), B, want in [((64, 64, 8), 8, 1), ((64, 64, 8), 4, 1), ((64, 64, 8), 2, 0),
                                      ((3, 16, 16), 8, 0), ((64, 32, 8), 8, 0), ((16, 64, 8), 8, 0)]:
            F = synth.conv_weights(1, "tcsel", co, ci, 3, 3, -128, 127)
            f = H.he_pack_filters_for_batch(p, dict(ci=ci, co=co, h=hw, w=hw), F, B)
            try:
                assert H.he_filters_tensor_core(f) == want, (ci, co, hw, B)
            finally:
                H.he_filters_destroy(f)


# (N, L, ci, co, hw, B, in_domain): K = G*s of 32, 64, 128, 256; s = 8 .. 64;
# 64 and 128 channels; odd and small batches (columns padded to 16)
TC_CASES = [
    (4096, 2, 64, 64, 8, 8, "coeff"),     # s = 32, G = 2, K = 64
    (4096, 2, 32, 64, 8, 4, "ntt"),       # s = 32, G = 1, K = 32
    (4096, 1, 128, 128, 8, 2, "coeff"),   # s = 32, G = 4, K = 128, two channel groups
    (4096, 2, 256, 64, 4, 1, "coeff"),    # s = 64, G = 4, K = 256
    (4096, 2, 64, 64, 20, 3, "coeff"),    # s = 8, G = 8, K = 64
    (8192, 3, 64, 128, 16, 8, "ntt"),     # s = 16, G = 4, K = 64, M = 512
]


@pytest.mark.parametrize("N,L,ci,co,hw,B,dom", TC_CASES)
def test_tensor_core_plan_matches_oracle(N, L, ci, co, hw, B, dom):
    H = U.he()
    torch = U.torch_cuda()
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=700 + ci + co + hw)
    ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_filters_for_batch(p, desc, F, 8)
        # a scalar-form call of another shape in the same plan
        f2 = H.he_pack_filters(p, dict(ci=3, co=16, h=16, w=16), synth.conv_weights(9, "o", 16, 3, 3, 3, -8, 7))
        try:
            assert H.he_filters_tensor_core(f) == 1
            x = _ntt_inputs(cts, ps, psis) if dom == "ntt" else cts
            lay2 = O.conv_layout(N, 3, 16, 16, 16)
            x2 = synth.residues(9, "o/x", (1, lay2["G"], 2, L, N), ps)
            ref2 = O.conv_layer(x2, synth.conv_weights(9, "o", 16, 3, 3, 3, -8, 7), ps, psis, lay2,
                                O.OUT_EXTRACTED, tier="ntt")
            d_in, d_out = U.to_dev(x), U.empty_dev(ref.shape)
            d_in2, d_out2 = U.to_dev(x2), U.empty_dev(ref2.shape)
            calls = [(f, d_in, H.HE_NTT if dom == "ntt" else H.HE_COEFF, d_out, B),
                     (f2, d_in2, H.HE_COEFF, d_out2, 1)]
            # the tensor-core kernel at every batch size (tc_min_batch = 1), then
            # batches below 4 on the bank's scalar-layout copy (split or fused form)
            for tmin in (1, 4):
                plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), tc_min_batch=tmin))
                try:
                    info = H.he_plan_query(plan, len(calls))
                    assert (info["form"][0] == 2) == (B >= tmin) and (info["tc_calls"] == 1) == (B >= tmin)
                    s = torch.cuda.current_stream()
                    for _ in range(2):  # repeatable: every word rewritten each run
                        d_out.fill_(-1)
                        d_out2.fill_(-1)
                        H.he_plan_run(plan, s)
                        H.he_sync(s)
                        H.he_plan_check(plan)
                        np.testing.assert_array_equal(U.from_dev(d_out).reshape(ref.shape), ref)
                        np.testing.assert_array_equal(U.from_dev(d_out2).reshape(ref2.shape), ref2)
                finally:
                    H.he_plan_destroy(plan)
        finally:
            H.he_filters_destroy(f)
            H.he_filters_destroy(f2)


@pytest.mark.parametrize("mode", ["HE_OUT_EXTRACTED", "HE_OUT_PER_CHANNEL", "HE_OUT_EXTRACTED_UNFOLDED"])
def test_single_calls_read_the_tensor_core_bank(mode):
    H = U.he()
    N, L, B = 4096, 2, 2
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, 64, 64, 8, 8, B, seed=77)
    omode = {"HE_OUT_EXTRACTED": O.OUT_EXTRACTED, "HE_OUT_PER_CHANNEL": O.OUT_PER_CHANNEL,
             "HE_OUT_EXTRACTED_UNFOLDED": O.OUT_EXTRACTED}[mode]
    ref = O.conv_layer(cts, F, ps, psis, lay, omode, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_filters_for_batch(p, desc, F, 8)
        try:
            assert H.he_filters_tensor_core(f) == 1
            got = U.run_conv(p, f, cts, getattr(H, mode), ref.shape[1])
            np.testing.assert_array_equal(got, ref)
        finally:
            H.he_filters_destroy(f)


def test_more_than_8_ciphertexts_take_the_scalar_form_on_a_tensor_core_bank():
    H = U.he()
    torch = U.torch_cuda()
    N, L, B = 4096, 1, 9
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, 64, 64, 8, 8, B, seed=78)
    ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_filters_for_batch(p, desc, F, 16)
        try:
            d_in, d_out = U.to_dev(cts), U.empty_dev(ref.shape)
            plan = H.he_plan_create([(f, d_in, H.HE_COEFF, d_out, B)])
            try:
                info = H.he_plan_query(plan, 1)
                assert info["tc_calls"] == 0 and info["fused_items"] > 0
                H.he_plan_run(plan, torch.cuda.current_stream())
                H.he_sync(torch.cuda.current_stream())
                np.testing.assert_array_equal(U.from_dev(d_out).reshape(ref.shape), ref)
            finally:
                H.he_plan_destroy(plan)
        finally:
            H.he_filters_destroy(f)


WIDE4_SHAPES = [(64, 64, 32), (64, 128, 32), (128, 128, 16), (128, 256, 16), (256, 256, 8)]


def test_wide4_batch8_tensor_core_equals_scalar_and_oracle():
    """The wide x4 layers at their full size (N = 16384, 6 limbs, B = 8): the
    tensor-core plan and the scalar kernels on the ordinary bank give the
    same words, every word of every limb equals the oracle's NTT tier, and
    sampled words its schoolbook dot products (an independent tier)."""
    H = U.he()
    torch = U.torch_cuda()
    N, L, B = 16384, 6, 8
    ps, psis = U.ring(N, L)
    rng = np.random.default_rng(11)
    with U.params(N, L) as p:
        for k, (ci, co, hw) in enumerate(WIDE4_SHAPES):
            _, _, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=800 + k)
            f_s = H.he_pack_filters(p, desc, F)
            f_t = H.he_pack_filters_for_batch(p, desc, F, B)
            try:
                assert H.he_filters_tensor_core(f_t) == 1
                scalar = U.run_conv(p, f_s, cts, H.HE_OUT_EXTRACTED, lay["H"])
                d_in, d_out = U.to_dev(cts), U.empty_dev(scalar.shape)
                plan = H.he_plan_create([(f_t, d_in, H.HE_COEFF, d_out, B)])
                try:
                    assert H.he_plan_query(plan, 1)["tc_calls"] == 1
                    H.he_plan_run(plan, torch.cuda.current_stream())
                    H.he_sync(torch.cuda.current_stream())
                    H.he_plan_check(plan)
                finally:
                    H.he_plan_destroy(plan)
                got = U.from_dev(d_out).reshape(scalar.shape)
                np.testing.assert_array_equal(got, scalar)
                ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
                np.testing.assert_array_equal(got, ref)
                picks = [(int(rng.integers(B)), int(rng.integers(lay["H"])), int(rng.integers(2)),
                          int(rng.integers(L)), int(rng.integers(N))) for _ in range(12)]
                np.testing.assert_array_equal(O.conv_layer_sampled(cts, F, ps, lay, picks),
                                              np.array([got[pk] for pk in picks], dtype=np.uint32))
            finally:
                H.he_filters_destroy(f_s)
                H.he_filters_destroy(f_t)
