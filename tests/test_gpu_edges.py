"""Edge cases at the limits of the path: the largest ring (N = 32768), the
most limbs (16), degenerate shapes (one input or output channel, a 1x1
image, 1x1 filters), the widest FC input (n_in = N: one row per weight
polynomial) and the masked step at N = 32768.  Every word against the
oracle (its NTT tier; on the largest cases one limb in full plus sampled
schoolbook words), through single calls and plans."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu
T = U.T


def _plan_and_single(H, p, f, cts, B, out_polys):
    torch = U.torch_cuda()
    single = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, out_polys)
    d_in, d_out = U.to_dev(cts), U.empty_dev(single.shape)
    plan = H.he_plan_create([(f, d_in, H.HE_COEFF, d_out, B)])
    try:
        H.he_plan_run(plan, torch.cuda.current_stream())
        H.he_sync(torch.cuda.current_stream())
        H.he_plan_check(plan)
    finally:
        H.he_plan_destroy(plan)
    got = U.from_dev(d_out).reshape(single.shape)
    np.testing.assert_array_equal(got, single)
    return got


# (N, L, ci, co, h, w, fh, pad, B)
CASES = [
    (32768, 2, 16, 32, 32, 32, 3, 1, 1),   # the largest ring
    (1024, 16, 3, 4, 4, 4, 3, 1, 2),       # the most limbs
    (2048, 3, 1, 5, 8, 8, 3, 1, 1),        # one input channel
    (2048, 3, 7, 1, 8, 8, 3, 1, 3),        # one output channel
    (1024, 2, 9, 6, 1, 1, 3, 1, 1),        # a 1x1 image
    (4096, 2, 40, 24, 6, 6, 1, 0, 2),      # 1x1 filters, no padding
]


@pytest.mark.parametrize("N,L,ci,co,h,w,fh,pad,B", CASES)
def test_conv_edge_cases(N, L, ci, co, h, w, fh, pad, B):
    H = U.he()
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, h, w, B, seed=N + L + ci + co, fh=fh, fw=fh, pad=pad)
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        got = _plan_and_single(H, p, f, cts, B, lay["H"])
    if N * L <= 2 * 8192:
        ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
        np.testing.assert_array_equal(got, ref)
    else:
        l = L - 1
        ref = O.conv_layer(np.ascontiguousarray(cts[:, :, :, l:l + 1]), F, [ps[l]], [psis[l]], lay, O.OUT_EXTRACTED,
                           tier="ntt")
        np.testing.assert_array_equal(got[:, :, :, l:l + 1], ref)
        rng = np.random.default_rng(N)
        picks = [(int(rng.integers(B)), int(rng.integers(lay["H"])), int(rng.integers(2)), int(rng.integers(L)),
                  int(rng.integers(N))) for _ in range(12)]
        np.testing.assert_array_equal(O.conv_layer_sampled(cts, F, ps, lay, picks),
                                      np.array([got[pk] for pk in picks], dtype=np.uint32))


def test_fc_with_the_widest_input():
    """n_in = N: one output row per weight polynomial (P = n_out)."""
    H = U.he()
    torch = U.torch_cuda()
    N, L, n_in, n_out, B = 1024, 2, 1024, 3, 2
    ps, psis = U.ring(N, L)
    lay = O.fc_layout(N, n_in, n_out)
    assert lay["P"] == n_out and lay["rows_per_poly"] == 1
    W = synth.fc_weights(7, "edge/W", n_out, n_in, -128, 127)
    Bv = synth.ints(7, "edge/B", (n_out,), -9, 9).astype(np.int32)
    ct = synth.residues(7, "edge/ct", (B, 2, L, N), ps)
    ref = O.fc_layer(ct, W, Bv, ps, psis, T, lay, O.OUT_EXTRACTED, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_fc(p, n_in, n_out, W, Bv)
        try:
            d_out = U.empty_dev(ref.shape)
            U.reserve(p, H.he_fc_workspace_bytes(p, B))
            H.he_fc_layer(p, f, U.to_dev(ct), H.HE_COEFF, d_out, H.HE_OUT_EXTRACTED, B, torch.cuda.current_stream())
            H.he_sync(torch.cuda.current_stream())
            np.testing.assert_array_equal(U.from_dev(d_out).reshape(ref.shape), ref)
            d_plan = U.empty_dev(ref.shape)
            plan = H.he_plan_create([(f, U.to_dev(ct), H.HE_COEFF, d_plan, B)])
            try:
                H.he_plan_run(plan, torch.cuda.current_stream())
                H.he_sync(torch.cuda.current_stream())
            finally:
                H.he_plan_destroy(plan)
            np.testing.assert_array_equal(U.from_dev(d_plan).reshape(ref.shape), ref)
        finally:
            H.he_filters_destroy(f)


def test_masked_step_on_the_largest_ring():
    H = U.he()
    torch = U.torch_cuda()
    N, L, ci, co, hw = 32768, 1, 32, 16, 16
    ps, psis = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    G, Hh = lay["G"], lay["H"]
    c0 = synth.residues(8, "edge/c0", (1, G, L, N), ps)
    sh = synth.ints(8, "edge/sh", (1, G, N), 0, T - 1).astype(np.uint32)
    rho = synth.ints(8, "edge/rho", (co, G, N), 0, T - 1).astype(np.uint32)
    shp = synth.ints(8, "edge/shp", (1, Hh, N), 0, T - 1).astype(np.uint32)
    F = synth.conv_weights(8, "edge/F", co, ci, 3, 3, -128, 127)
    ref = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_masked(p, dict(ci=ci, co=co, h=hw, w=hw), F, rho)
        try:
            d_out = U.empty_dev(ref.shape)
            H.he_conv_layer_masked(p, f, U.to_dev(c0), U.to_dev(sh), U.to_dev(shp), H.HE_COEFF, d_out, 1,
                                   torch.cuda.current_stream())
            H.he_sync(torch.cuda.current_stream())
            np.testing.assert_array_equal(U.from_dev(d_out).reshape(ref.shape), ref)
            d_plan = U.empty_dev(ref.shape)
            plan = H.he_plan_create([(f, U.to_dev(c0), H.HE_COEFF, d_plan, 1, U.to_dev(sh), U.to_dev(shp))])
            try:
                H.he_plan_run(plan, torch.cuda.current_stream())
                H.he_sync(torch.cuda.current_stream())
                H.he_plan_check(plan)
            finally:
                H.he_plan_destroy(plan)
            np.testing.assert_array_equal(U.from_dev(d_plan).reshape(ref.shape), ref)
        finally:
            H.he_filters_destroy(f)
