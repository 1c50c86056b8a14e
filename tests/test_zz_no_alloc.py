"""he_conv_layer_noalloc: the Conv layer call that allocates nothing.

It must give, word for word, what he_conv_layer gives on the same inputs, on
consecutive calls that reuse its fixed scratch, and reject inputs larger than
that scratch before launching anything.  The file is named to run last, so
that it also runs after every other GPU test in one process.
"""

from __future__ import annotations

import numpy as np
import pytest

import _gpu_helpers as U

pytestmark = pytest.mark.gpu

SCRATCH_WORDS = 2 * 1024 * 1024


def _both(H, p, f, cts, mode, out_polys, in_domain):
    torch = U.torch_cuda()
    B, G, _, L, N = cts.shape
    st = torch.cuda.current_stream()
    d_in = U.to_dev(cts)
    ref = U.empty_dev((B, out_polys, 2, L, N))
    got = U.empty_dev((B, out_polys, 2, L, N), fill=0x5A5A5A5A)
    U.reserve(p, cts.size * 4)  # he_conv_layer's workspace, sized before its call
    H.he_conv_layer(p, f, d_in, in_domain, ref, mode, B, st)
    H.he_conv_layer_noalloc(p, f, d_in, in_domain, got, mode, B, st)
    H.he_sync(st)
    return U.from_dev(ref), U.from_dev(got)


@pytest.mark.parametrize("case", [
    # N, L, ci, co, h, w, B
    (1024, 3, 16, 8, 8, 8, 2),
    (8192, 3, 16, 16, 32, 32, 1),
    (4096, 2, 40, 12, 8, 8, 3),
])
def test_noalloc_matches_conv_layer_on_consecutive_calls(case):
    H = U.he()
    N, L, ci, co, h, w, B = case
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, h, w, B, seed=21)
    cts2 = U.synth.residues(22, "noalloc/second", cts.shape, ps)
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        for x in (cts, cts2):  # two calls in a row through the same scratch
            for mode, polys in ((H.HE_OUT_EXTRACTED, lay["H"]), (H.HE_OUT_PER_CHANNEL, co)):
                ref, got = _both(H, p, f, x, mode, polys, H.HE_COEFF)
                np.testing.assert_array_equal(got, ref)
        ref, got = _both(H, p, f, cts, H.HE_OUT_EXTRACTED, lay["H"], H.HE_NTT)
        np.testing.assert_array_equal(got, ref)


def test_noalloc_needs_no_workspace_and_allocates_nothing():
    """On fresh params whose workspace only covers one ciphertext, a call of
    three runs through the scratch alone (he_conv_layer refuses the same call
    until it is reserved), and a second call leaves the device's free memory
    unchanged."""
    H = U.he()
    torch = U.torch_cuda()
    N, L, ci, co, h, w, B = 1024, 3, 16, 8, 8, 8, 3
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, h, w, B, seed=25)
    cts2 = U.synth.residues(26, "noalloc/fresh2", cts.shape, ps)
    st = torch.cuda.current_stream()
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        d_in, d_in2 = U.to_dev(cts), U.to_dev(cts2)
        got = U.empty_dev((B, lay["H"], 2, L, N), fill=0x5A5A5A5A)
        got2 = U.empty_dev((B, lay["H"], 2, L, N), fill=0x5A5A5A5A)
        H.he_conv_layer_noalloc(p, f, d_in, H.HE_COEFF, got, H.HE_OUT_EXTRACTED, B, st)  # first call: set-up
        H.he_sync(st)
        free0 = torch.cuda.mem_get_info()[0]
        H.he_conv_layer_noalloc(p, f, d_in2, H.HE_COEFF, got2, H.HE_OUT_EXTRACTED, B, st)
        H.he_sync(st)
        assert torch.cuda.mem_get_info()[0] == free0
        ref = U.empty_dev((B, lay["H"], 2, L, N))
        with pytest.raises(H.HEError) as ei:
            H.he_conv_layer(p, f, d_in, H.HE_COEFF, ref, H.HE_OUT_EXTRACTED, B, st)
        assert ei.value.status == H.HE_ERR_NOMEM
        U.reserve(p, cts.size * 4)
        for x, g in ((d_in, got), (d_in2, got2)):
            H.he_conv_layer(p, f, x, H.HE_COEFF, ref, H.HE_OUT_EXTRACTED, B, st)
            H.he_sync(st)
            np.testing.assert_array_equal(U.from_dev(g), U.from_dev(ref))


def test_noalloc_matches_the_oracle():
    H = U.he()
    ps, psis, lay, cts, F, desc = U.conv_case(2048, 2, 5, 6, 8, 8, 2, seed=23)
    want = U.O.conv_layer(cts, F, ps, psis, lay, U.O.OUT_EXTRACTED)
    with U.params(2048, 2) as p, U.conv_bank(p, desc, F) as f:
        _, got = _both(H, p, f, cts, H.HE_OUT_EXTRACTED, lay["H"], H.HE_COEFF)
    np.testing.assert_array_equal(got.reshape(want.shape), want)


def test_noalloc_rejects_inputs_above_its_scratch():
    H = U.he()
    N, L, ci, co, h, w = 16384, 6, 3, 4, 16, 16
    lay = U.O.conv_layout(N, ci, co, h, w)
    B = SCRATCH_WORDS // (lay["G"] * 2 * L * N) + 1
    assert B * lay["G"] * 2 * L * N > SCRATCH_WORDS
    F = U.synth.conv_weights(24, "noalloc/big", co, ci, 3, 3, -8, 7)
    torch = U.torch_cuda()
    with U.params(N, L) as p, U.conv_bank(p, dict(ci=ci, co=co, h=h, w=w), F) as f:
        d_in = U.empty_dev((B, lay["G"], 2, L, N), fill=0)
        d_out = U.empty_dev((B, lay["H"], 2, L, N), fill=0)
        with pytest.raises(H.HEError) as ei:
            H.he_conv_layer_noalloc(p, f, d_in, H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B,
                                    torch.cuda.current_stream())
        assert ei.value.status == H.HE_ERR_ARG and "scratch" in str(ei.value)
        # one fewer ciphertext fits and runs
        B1 = B - 1
        H.he_conv_layer_noalloc(p, f, d_in, H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B1,
                                torch.cuda.current_stream())
        H.he_sync(torch.cuda.current_stream())
