"""GPU parity: every output word of the CUDA path, called through the C ABI,
equals the oracle's (bit-exact: the work is integer arithmetic mod q_l).

Sizes: small rings that span several tiles with ragged tails, the single
Conv config (N = 2048), every distinct plain-20 layer shape at N = 8192 with
3 limbs, and wide layers at N = 16384 with 6 limbs and B = 8.  Edge cases:
interleave s = 1, 2 and 128, c_o < s, a partly filled last output
polynomial, several input groups, inputs already in the NTT domain, and
argument errors."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

import _gpu_helpers as U

pytestmark = pytest.mark.gpu

MODES = ["extracted", "unfolded", "per_channel"]


def _mode(H, name):
    return {"extracted": H.HE_OUT_EXTRACTED, "unfolded": H.HE_OUT_EXTRACTED_UNFOLDED,
            "per_channel": H.HE_OUT_PER_CHANNEL}[name]


def _ref_conv(cts, F, ps, psis, lay, mode_name, tier="ntt"):
    m = O.OUT_PER_CHANNEL if mode_name == "per_channel" else O.OUT_EXTRACTED
    return O.conv_layer(cts, F, ps, psis, lay, m, tier=tier)


# ----------------------------------------------------------------------------
# NTT
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N,L,count", [(64, 1, 3), (1024, 2, 2), (2048, 1, 5), (8192, 3, 4),
                                       (16384, 6, 2), (32768, 1, 2)])
def test_forward_and_inverse_ntt_match_oracle(N, L, count):
    H = U.he()
    ps, psis = U.ring(N, L)
    a = synth.residues(N, "ntt", (count, L, N), ps)
    with U.params(N, L) as p:
        d = U.to_dev(a)
        out = U.empty_dev(a.shape)
        H.he_ntt_forward(p, d, out, count)
        H.he_sync()
        got = U.from_dev(out).reshape(a.shape)
        for l in range(L):
            np.testing.assert_array_equal(got[:, l], O.ntt_fwd(a[:, l], ps[l], psis[l]))
        back = U.empty_dev(a.shape)
        H.he_ntt_inverse(p, out, back, count)
        H.he_ntt_forward(p, back, back, count)      # in place
        H.he_ntt_inverse(p, back, back, count)
        H.he_sync()
        np.testing.assert_array_equal(U.from_dev(back).reshape(a.shape), a)


# ----------------------------------------------------------------------------
# Conv: small rings, every mode, edge cases
# ----------------------------------------------------------------------------

SMALL = [
    # N, L, ci, co, h, w, B, fh, fw, pad       (s, G, H) noted
    (256, 1, 3, 4, 4, 4, 1, 3, 3, 1),        # s=4 G=1 H=1
    (256, 2, 8, 2, 4, 4, 2, 3, 3, 1),        # s=4, c_o=2 < s: offsets spread by 2
    (512, 1, 16, 10, 4, 4, 3, 3, 3, 1),      # s=8, G=2, H=2 with a ragged last output poly
    (1024, 2, 5, 7, 6, 5, 1, 3, 3, 1),       # odd shapes
    (1024, 1, 1, 3, 8, 8, 2, 3, 3, 1),       # s = 1
    (256, 1, 16, 16, 8, 8, 1, 3, 3, 1),      # s = 2 (P = 100), G = 8
    (512, 2, 200, 130, 2, 2, 1, 2, 1, 0),    # s = 128 (P = 4), G = 2, H = 2 ragged
    (64, 1, 4, 4, 2, 2, 1, 2, 1, 0),         # the paper's tiny example, N = 64
    (2048, 1, 32, 64, 4, 4, 2, 3, 3, 1),     # s = 32, H = 2
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", SMALL, ids=[f"N{c[0]}_ci{c[2]}_co{c[3]}" for c in SMALL])
def test_conv_small_rings_all_modes(case, mode):
    H = U.he()
    N, L, ci, co, h, w, B, fh, fw, pad = case
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, h, w, B, seed=7, fh=fh, fw=fw, pad=pad)
    ref = _ref_conv(cts, F, ps, psis, lay, mode)
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        got = U.run_conv(p, f, cts, _mode(H, mode), ref.shape[1])
    np.testing.assert_array_equal(got, ref)


def test_conv_small_schoolbook_reference():
    H = U.he()
    ps, psis, lay, cts, F, desc = U.conv_case(256, 2, 5, 6, 4, 4, 2, seed=8)
    ref = _ref_conv(cts, F, ps, psis, lay, "extracted", tier="schoolbook")
    with U.params(256, 2) as p, U.conv_bank(p, desc, F) as f:
        got = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"])
    np.testing.assert_array_equal(got, ref)


def test_conv_inputs_in_ntt_domain():
    H = U.he()
    ps, psis, lay, cts, F, desc = U.conv_case(1024, 3, 16, 8, 8, 8, 2, seed=9)
    ref = _ref_conv(cts, F, ps, psis, lay, "extracted")
    with U.params(1024, 3) as p, U.conv_bank(p, desc, F) as f:
        got = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"], in_domain=H.HE_NTT)
    np.testing.assert_array_equal(got, ref)


# ----------------------------------------------------------------------------
# The single Conv config: N = 2048, one 30-bit prime, 3x16x16 input, 4 outputs
# ----------------------------------------------------------------------------

def test_conv1_config_bit_exact_and_decrypts():
    H = U.he()
    N, ci, co, h, w = 2048, 3, 4, 16, 16
    ps, psis = U.ring(N, 1)
    lay = O.conv_layout(N, ci, co, h, w)
    F = synth.conv_weights(1, "conv1/F", co, ci, 3, 3, -8, 7)
    I = synth.ints(1, "conv1/I", (ci, h, w), -8, 7)
    desc = dict(ci=ci, co=co, h=h, w=w)
    # uniform ciphertext, every mode, schoolbook reference
    cts = synth.residues(1, "conv1/ct", (1, 1, 2, 1, N), ps)
    with U.params(N, 1) as p, U.conv_bank(p, desc, F) as f:
        for mode in MODES:
            ref = _ref_conv(cts, F, ps, psis, lay, mode, tier="schoolbook")
            got = U.run_conv(p, f, cts, _mode(H, mode), ref.shape[1])
            np.testing.assert_array_equal(got, ref)
        # a real RLWE encryption: ternary secret, centered-binomial error (eta 3)
        s = synth.ternary(1, "conv1/s", N)
        a = synth.residues(1, "conv1/a", (1, N), ps)
        e = synth.cbd(1, "conv1/e", N, 3)
        ct = O.encrypt_sk(O.pack_input(I, lay)[0], s, a, e, ps, U.T)[None, None]
        y = U.run_conv(p, f, ct, H.HE_OUT_PER_CHANNEL, co)
    want = O.centered(O.direct_conv(I, F, 1), U.T)
    for n in range(co):
        m = O.decrypt(y[0, n], s, ps, U.T)
        got = np.array([[m[O.output_slot(lay, n, k, l)[1]] for l in range(w)] for k in range(h)])
        np.testing.assert_array_equal(got, want[n])


# ----------------------------------------------------------------------------
# plain-20 layer shapes at N = 8192, 3 limbs, B = 1 (every word vs the CPU
# NTT tier, plus sampled coefficients by schoolbook dot products)
# ----------------------------------------------------------------------------

PLAIN20_SHAPES = [(3, 16, 32), (16, 16, 32), (16, 32, 32), (32, 32, 16), (32, 64, 16), (64, 64, 8)]


@pytest.mark.parametrize("ci,co,hw", PLAIN20_SHAPES)
def test_plain20_layer_shapes_full_size(ci, co, hw):
    H = U.he()
    N, L = 8192, 3
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, 1, seed=20)
    ref = _ref_conv(cts, F, ps, psis, lay, "extracted")
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        got = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"])
    np.testing.assert_array_equal(got, ref)
    rng = np.random.default_rng(ci * 1000 + co)
    picks = [(0, int(rng.integers(lay["H"])), int(rng.integers(2)), int(rng.integers(L)),
              int(rng.integers(N))) for _ in range(24)]
    np.testing.assert_array_equal(O.conv_layer_sampled(cts, F, ps, lay, picks),
                                  np.array([got[pk] for pk in picks], dtype=np.uint32))


# ----------------------------------------------------------------------------
# wide layers: N = 16384, 6 limbs, B = 8
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("ci,co,hw", [(256, 256, 8), (3, 64, 32), (64, 128, 32)])
def test_wide_layers_batch8(ci, co, hw):
    H = U.he()
    N, L, B = 16384, 6, 8
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=40)
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        got = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"])
    # every word of two limbs against the CPU NTT tier, sampled words of all
    for l in (0, L - 1):
        ref = O.conv_layer(np.ascontiguousarray(cts[:, :, :, l:l + 1]), F, [ps[l]], [psis[l]],
                           lay, O.OUT_EXTRACTED, tier="ntt")
        np.testing.assert_array_equal(got[:, :, :, l:l + 1], ref)
    rng = np.random.default_rng(co)
    picks = [(int(rng.integers(B)), int(rng.integers(lay["H"])), int(rng.integers(2)),
              int(rng.integers(L)), int(rng.integers(N))) for _ in range(16)]
    np.testing.assert_array_equal(O.conv_layer_sampled(cts, F, ps, lay, picks),
                                  np.array([got[pk] for pk in picks], dtype=np.uint32))


# ----------------------------------------------------------------------------
# FC
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N,L,n_in,n_out,B,bias", [
    (8192, 3, 64, 10, 1, True), (4096, 2, 64, 100, 2, True), (16384, 6, 256, 100, 8, False),
    (512, 1, 6, 40, 3, True), (256, 2, 64, 10, 1, False)])
def test_fc_matches_oracle(N, L, n_in, n_out, B, bias):
    H = U.he()
    ps, psis = U.ring(N, L)
    lay = O.fc_layout(N, n_in, n_out)
    W = synth.fc_weights(N, "fcW", n_out, n_in, -128, 127)
    Bv = synth.ints(N, "fcB", (n_out,), -30000, 30000) if bias else None
    ct = synth.residues(N, "fcct", (B, 2, L, N), ps)
    with U.params(N, L) as p, U.fc_bank(p, n_in, n_out, W, Bv) as f:
        for mode, omode in ((H.HE_OUT_EXTRACTED, O.OUT_EXTRACTED), (H.HE_OUT_PER_CHANNEL, O.OUT_PER_CHANNEL)):
            got = U.run_fc(p, f, ct, mode, lay["P"])
            ref = O.fc_layer(ct, W, Bv, ps, psis, U.T, lay, omode, tier="ntt")
            np.testing.assert_array_equal(got, ref)


def test_fc_encrypt_eval_decrypt():
    H = U.he()
    N, L, n_in, n_out = 8192, 3, 64, 10
    ps, psis = U.ring(N, L)
    lay = O.fc_layout(N, n_in, n_out)
    W = synth.fc_weights(5, "W", n_out, n_in, -128, 127)
    I = synth.ints(5, "I", (n_in,), -100, 100)
    Bv = synth.ints(5, "B", (n_out,), -1000, 1000)
    s = synth.ternary(5, "s", N)
    a = synth.residues(5, "a", (L, N), ps)
    ct = O.encrypt_sk(O.pack_fc_input(I, lay), s, a, synth.cbd(5, "e", N), ps, U.T)[None]
    with U.params(N, L) as p, U.fc_bank(p, n_in, n_out, W, Bv) as f:
        y = U.run_fc(p, f, ct, H.HE_OUT_PER_CHANNEL, lay["P"])
    m = O.decrypt(y[0, 0], s, ps, U.T)
    np.testing.assert_array_equal(m[:n_out], O.centered(W.astype(np.int64) @ I + Bv, U.T))


# ----------------------------------------------------------------------------
# argument errors, workspace growth, repeatability
# ----------------------------------------------------------------------------

def test_argument_errors_and_larger_batches():
    H = U.he()
    torch = U.torch_cuda()
    ps, psis, lay, cts, F, desc = U.conv_case(1024, 1, 8, 8, 6, 6, 4, seed=11)
    with U.params(1024, 1) as p, U.conv_bank(p, desc, F) as f:
        buf = U.empty_dev((8, lay["G"] * 2 * 1024 * 8))
        with pytest.raises(H.HEError) as ei:   # overlapping input and output
            H.he_conv_layer(p, f, buf, H.HE_COEFF, buf, H.HE_OUT_EXTRACTED, 1)
        assert ei.value.status == H.HE_ERR_ARG
        with pytest.raises(H.HEError) as ei:   # misaligned
            H.he_conv_layer(p, f, buf.data_ptr() + 4, H.HE_COEFF, U.empty_dev((1 << 16,)),
                            H.HE_OUT_EXTRACTED, 1)
        assert ei.value.status == H.HE_ERR_ARG
        with pytest.raises(H.HEError) as ei:   # conv bank given to the FC entry point
            H.he_fc_layer(p, f, buf, H.HE_COEFF, U.empty_dev((1 << 16,)), H.HE_OUT_EXTRACTED, 1)
        assert ei.value.status == H.HE_ERR_ARG
        with pytest.raises(H.HEError) as ei:
            H.he_conv_layer(p, f, buf, 7, U.empty_dev((1 << 16,)), H.HE_OUT_EXTRACTED, 1)
        assert ei.value.status == H.HE_ERR_ARG
        # B = 1, then B = 4 with its workspace reserved; results stay exact and repeatable
        ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
        got1 = U.run_conv(p, f, cts[:1], H.HE_OUT_EXTRACTED, lay["H"])
        np.testing.assert_array_equal(got1, ref[:1])
        got4 = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"])
        got4b = U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"])
        np.testing.assert_array_equal(got4, ref)
        np.testing.assert_array_equal(got4b, ref)
    torch.cuda.synchronize()


# ----------------------------------------------------------------------------
# plans: many calls in one launch pair, bit-exact against the oracle
# ----------------------------------------------------------------------------

def _plan_case(H, p, N, L, shape, B, seed, fc=False):
    ps, psis = U.ring(N, L)
    if fc:
        n_in, n_out = shape
        lay = O.fc_layout(N, n_in, n_out)
        W = synth.fc_weights(seed, "pW", n_out, n_in, -128, 127)
        Bv = synth.ints(seed, "pB", (n_out,), -999, 999)
        ct = synth.residues(seed, "pct", (B, 2, L, N), ps)
        ref = O.fc_layer(ct, W, Bv, ps, psis, U.T, lay, O.OUT_EXTRACTED, tier="ntt")
        f = H.he_pack_fc(p, n_in, n_out, W, Bv)
        return f, ct, ref
    ci, co, hw = shape
    _, _, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=seed)
    ref = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
    f = H.he_pack_filters(p, desc, F)
    return f, cts, ref


def test_plan_mixed_rings_and_shapes_bit_exact():
    """A plan over independent calls with N in {1024, 2048, 4096}, 1-3 limbs,
    B in {1, 2, 8}, Conv shapes with s = 2 .. 64 and FC layers (split over 2
    and 3 weight polynomials), some inputs already in the NTT domain; built
    with the default tuning and with fc_direct = 2, which computes the window
    of every coefficient-domain FC call directly (the last call's third block
    ragged)."""
    H = U.he()
    torch = U.torch_cuda()
    specs = [(1024, 2, (16, 16, 8), 1, False), (2048, 1, (3, 4, 16), 1, False),
             (4096, 3, (16, 16, 32), 1, False), (4096, 2, (64, 100), 1, True),
             (2048, 3, (32, 64, 4), 2, False), (1024, 1, (64, 10), 2, True),
             (4096, 2, (8, 16, 8), 8, False), (2048, 2, (200, 20), 2, True)]
    pars = {}
    calls, refs, outs, keep = [], [], [], []
    try:
        for k, (N, L, shape, B, fc) in enumerate(specs):
            if (N, L) not in pars:
                pars[(N, L)] = H.he_params_create(N, L, None, U.T, 0)
            p = pars[(N, L)]
            f, x, ref = _plan_case(H, p, N, L, shape, B, seed=100 + k, fc=fc)
            dom = H.HE_NTT if k % 3 == 2 else H.HE_COEFF
            if dom == H.HE_NTT:
                ps, psis = U.ring(N, L)
                x = x.copy()
                for l in range(L):
                    x[..., l, :] = O.ntt_fwd(np.ascontiguousarray(x[..., l, :]), ps[l], psis[l])
            d_in = U.to_dev(x)
            d_out = U.empty_dev(ref.shape)
            keep += [d_in, d_out]
            calls.append((f, d_in, dom, d_out, B))
            refs.append(ref)
            outs.append(d_out)
        for fc_direct in (1, 2):
            plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), fc_direct=fc_direct))
            try:
                form = H.he_plan_query(plan, len(calls))["form"]
                if fc_direct == 2:
                    assert form[3] == 3 and form[7] == 3   # the coefficient-domain FC calls
                s = torch.cuda.current_stream()
                for _ in range(2):           # repeatable: every word rewritten each run
                    for o in outs:
                        o.fill_(-1)
                    H.he_plan_run(plan, s)
                    H.he_sync(s)
                    H.he_plan_check(plan)
                    for o, ref in zip(outs, refs):
                        np.testing.assert_array_equal(U.from_dev(o).reshape(ref.shape), ref)
            finally:
                H.he_plan_destroy(plan)
    finally:
        for c in calls:
            H.he_filters_destroy(c[0])
        for p in pars.values():
            H.he_params_destroy(p)


def test_plan_captured_in_cuda_graph_matches_single_calls():
    H = U.he()
    torch = U.torch_cuda()
    N, L = 8192, 3
    with U.params(N, L) as p:
        shapes = [(3, 16, 32), (16, 32, 32), (64, 64, 8)]
        banks, calls, singles = [], [], []
        for k, sh in enumerate(shapes):
            ps, psis, lay, cts, F, desc = U.conv_case(N, L, sh[0], sh[1], sh[2], sh[2], 1, seed=200 + k)
            f = H.he_pack_filters(p, desc, F)
            banks.append(f)
            singles.append(U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"]))
            d_in, d_out = U.to_dev(cts), U.empty_dev(singles[-1].shape)
            calls.append((f, d_in, H.HE_COEFF, d_out, 1))
        plan = H.he_plan_create(calls)
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                H.he_plan_run(plan, s)          # warm-up outside capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                H.he_plan_run(plan, s)
            for c in calls:
                c[3].fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            for c, ref in zip(calls, singles):
                np.testing.assert_array_equal(U.from_dev(c[3]).reshape(ref.shape), ref)
        finally:
            H.he_plan_destroy(plan)
            for f in banks:
                H.he_filters_destroy(f)


def test_plan_rejects_overlapping_outputs():
    H = U.he()
    ps, psis, lay, cts, F, desc = U.conv_case(1024, 1, 8, 8, 6, 6, 1, seed=12)
    with U.params(1024, 1) as p, U.conv_bank(p, desc, F) as f:
        d_in = U.to_dev(cts)
        d_out = U.empty_dev((lay["H"] * 2 * 1024,))
        with pytest.raises(H.HEError) as ei:
            H.he_plan_create([(f, d_in, H.HE_COEFF, d_out, 1), (f, d_in, H.HE_COEFF, d_out, 1)])
        assert ei.value.status == H.HE_ERR_ARG
        with pytest.raises(H.HEError) as ei:
            H.he_plan_create([(f, d_in, H.HE_COEFF, d_in, 1)])
        assert ei.value.status == H.HE_ERR_ARG


def test_plan_split_form_plain20_shapes_bit_exact():
    """Every distinct plain-20 layer shape at N = 8192 with 3 limbs, B = 1
    (the split MAC + finishing kernels) and the FC layer, in one plan,
    against the oracle's NTT tier; the plan's status word stays clear."""
    H = U.he()
    torch = U.torch_cuda()
    N, L = 8192, 3
    ps, psis = U.ring(N, L)
    with U.params(N, L) as p:
        calls, refs, banks = [], [], []
        for k, (ci, co, hw) in enumerate(PLAIN20_SHAPES):
            _, _, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, 1, seed=300 + k)
            refs.append(O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt"))
            f = H.he_pack_filters(p, desc, F)
            banks.append(f)
            calls.append((f, U.to_dev(cts), H.HE_COEFF, U.empty_dev(refs[-1].shape), 1))
        f, ct, ref = _plan_case(H, p, N, L, (64, 10), 1, seed=399, fc=True)
        banks.append(f)
        refs.append(ref)
        calls.append((f, U.to_dev(ct), H.HE_COEFF, U.empty_dev(ref.shape), 1))
        plan = H.he_plan_create(calls)
        try:
            info = H.he_plan_query(plan, len(calls))
            assert info["split"] == [True] * len(PLAIN20_SHAPES) + [False]
            assert info["split_calls"] == len(PLAIN20_SHAPES)
            assert info["kernels_per_run"] == 3        # NTT (and the FC window), MAC, finish
            assert info["fc_items"] > 0 and info["fused_items"] == 0
            s = torch.cuda.current_stream()
            # the whole run, then the same run in phases 0 + 1 and 0 + 2 + 3
            for phases in (None, (H.HE_PHASE_NTT, H.HE_PHASE_REST),
                           (H.HE_PHASE_NTT, H.HE_PHASE_MAC, H.HE_PHASE_FINISH)):
                for c in calls:
                    c[3].fill_(-1)
                if phases is None:
                    H.he_plan_run(plan, s)
                else:
                    for ph in phases:
                        H.he_plan_run_phase(plan, ph, s)
                H.he_sync(s)
                H.he_plan_check(plan)
                for c, ref in zip(calls, refs):
                    np.testing.assert_array_equal(U.from_dev(c[3]).reshape(ref.shape), ref)
            H.he_plan_run_phase(plan, H.HE_PHASE_RESCALE, s)   # no call asks for a rescale: nothing runs
            H.he_sync(s)
            for bad in (-1, 6):
                with pytest.raises(H.HEError):
                    H.he_plan_run_phase(plan, bad, s)
        finally:
            H.he_plan_destroy(plan)
            for f in banks:
                H.he_filters_destroy(f)


# ----------------------------------------------------------------------------
# the wide x4 network (N = 16384, 6 limbs, B = 8) through one plan: every
# distinct Conv shape and the FC layer; every word equals the single-call
# path, sampled words equal the oracle
# ----------------------------------------------------------------------------

WIDE4_SHAPES = [(3, 64, 32), (64, 64, 32), (64, 128, 32), (128, 128, 16), (128, 256, 16), (256, 256, 8)]


def test_plan_wide4_batch8_matches_single_calls_and_oracle():
    H = U.he()
    torch = U.torch_cuda()
    N, L, B = 16384, 6, 8
    ps, psis = U.ring(N, L)
    with U.params(N, L) as p:
        calls, singles, banks, cases = [], [], [], []
        for k, (ci, co, hw) in enumerate(WIDE4_SHAPES):
            _, _, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=500 + k)
            f = H.he_pack_filters(p, desc, F)
            banks.append(f)
            singles.append(U.run_conv(p, f, cts, H.HE_OUT_EXTRACTED, lay["H"]))
            calls.append((f, U.to_dev(cts), H.HE_COEFF, U.empty_dev(singles[-1].shape), B))
            cases.append((cts, F, lay))
        fc_f, fc_ct, fc_ref = _plan_case(H, p, N, L, (256, 100), B, seed=599, fc=True)
        banks.append(fc_f)
        calls.append((fc_f, U.to_dev(fc_ct), H.HE_COEFF, U.empty_dev(fc_ref.shape), B))
        plan = H.he_plan_create(calls)
        try:
            info = H.he_plan_query(plan, len(calls))
            assert info["split_calls"] == 0  # B = 8: every Conv call takes the fused form
            s = torch.cuda.current_stream()
            H.he_plan_run(plan, s)
            H.he_sync(s)
            H.he_plan_check(plan)
            rng = np.random.default_rng(7)
            for c, ref, (cts, F, lay) in zip(calls, singles, cases):
                got = U.from_dev(c[3]).reshape(ref.shape)
                np.testing.assert_array_equal(got, ref)
                picks = [(int(rng.integers(B)), int(rng.integers(lay["H"])), int(rng.integers(2)),
                          int(rng.integers(L)), int(rng.integers(N))) for _ in range(12)]
                np.testing.assert_array_equal(O.conv_layer_sampled(cts, F, ps, lay, picks),
                                              np.array([got[pk] for pk in picks], dtype=np.uint32))
            np.testing.assert_array_equal(U.from_dev(calls[-1][3]).reshape(fc_ref.shape), fc_ref)
        finally:
            H.he_plan_destroy(plan)
            for f in banks:
                H.he_filters_destroy(f)
