"""The layer calls never allocate: their workspace is sized at model load.

A packed bank reserves the workspace of one call at the batch it was packed
for; a call that needs more fails with HE_ERR_NOMEM before anything is
launched, and runs bit-exact once he_params_reserve has sized the workspace.
"""

from __future__ import annotations

import numpy as np
import pytest

import _gpu_helpers as U

pytestmark = pytest.mark.gpu

FILL = 0x5A5A5A5A


def test_conv_call_above_the_reserved_workspace_fails_cleanly_then_runs_after_reserve():
    H = U.he()
    torch = U.torch_cuda()
    st = torch.cuda.current_stream()
    N, L, B = 2048, 2, 3
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, 5, 6, 8, 8, B, seed=31)
    want = U.O.conv_layer(cts, F, ps, psis, lay, U.O.OUT_EXTRACTED)
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        assert H.he_conv_workspace_bytes(p, desc, B) == cts.size * 4
        d_in = U.to_dev(cts)
        d_out = U.empty_dev(want.shape, fill=FILL)
        with pytest.raises(H.HEError) as ei:
            H.he_conv_layer(p, f, d_in, H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B, st)
        assert ei.value.status == H.HE_ERR_NOMEM and "he_params_reserve" in str(ei.value)
        H.he_sync(st)
        assert (U.from_dev(d_out) == FILL).all()  # nothing was launched
        # one ciphertext fits the workspace the bank reserved at model load
        one = U.empty_dev((1,) + want.shape[1:])
        H.he_conv_layer(p, f, U.to_dev(cts[:1]), H.HE_COEFF, one, H.HE_OUT_EXTRACTED, 1, st)
        H.he_sync(st)
        np.testing.assert_array_equal(U.from_dev(one).reshape(want[:1].shape), want[:1])
        H.he_params_reserve(p, H.he_conv_workspace_bytes(p, desc, B))
        free0 = torch.cuda.mem_get_info()[0]
        H.he_conv_layer(p, f, d_in, H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B, st)
        H.he_sync(st)
        assert torch.cuda.mem_get_info()[0] == free0  # the call allocated nothing
        np.testing.assert_array_equal(U.from_dev(d_out).reshape(want.shape), want)


def test_fc_call_above_the_reserved_workspace_fails_cleanly_then_runs_after_reserve():
    H = U.he()
    torch = U.torch_cuda()
    st = torch.cuda.current_stream()
    N, L, B, n_in, n_out = 1024, 2, 2, 64, 10
    ps, psis = U.ring(N, L)
    lay = U.O.fc_layout(N, n_in, n_out)
    W = U.synth.fc_weights(32, "ws/W", n_out, n_in, -128, 127)
    bias = U.synth.ints(32, "ws/b", (n_out,), -99, 99).astype(np.int32)
    ct = U.synth.residues(32, "ws/ct", (B, 2, L, N), ps)
    want = U.O.fc_layer(ct, W, bias, ps, psis, U.T, lay, U.O.OUT_EXTRACTED, tier="ntt")
    with U.params(N, L) as p, U.fc_bank(p, n_in, n_out, W, bias) as f:
        assert H.he_fc_workspace_bytes(p, B) == ct.size * 4
        d_out = U.empty_dev(want.shape, fill=FILL)
        with pytest.raises(H.HEError) as ei:
            H.he_fc_layer(p, f, U.to_dev(ct), H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B, st)
        assert ei.value.status == H.HE_ERR_NOMEM
        H.he_sync(st)
        assert (U.from_dev(d_out) == FILL).all()
        H.he_params_reserve(p, H.he_fc_workspace_bytes(p, B))
        H.he_fc_layer(p, f, U.to_dev(ct), H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B, st)
        H.he_sync(st)
        np.testing.assert_array_equal(U.from_dev(d_out).reshape(want.shape), want)


def test_bank_packed_for_a_batch_reserves_that_batch():
    H = U.he()
    torch = U.torch_cuda()
    st = torch.cuda.current_stream()
    N, L, B = 1024, 2, 4
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, 16, 8, 8, 8, B, seed=33)
    want = U.O.conv_layer(cts, F, ps, psis, lay, U.O.OUT_EXTRACTED)
    with U.params(N, L) as p:
        f = H.he_pack_filters_for_batch(p, desc, F, B)
        try:
            d_out = U.empty_dev(want.shape)
            H.he_conv_layer(p, f, U.to_dev(cts), H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B, st)
            H.he_sync(st)
            np.testing.assert_array_equal(U.from_dev(d_out).reshape(want.shape), want)
        finally:
            H.he_filters_destroy(f)
