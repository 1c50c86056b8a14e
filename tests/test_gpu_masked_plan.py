"""Masked (server) and client banks in plans: every call of a mixed plan
must write the words of its single-call entry point (he_conv_layer_masked,
he_fc_layer_masked, he_conv_client, he_fc_client, he_conv_layer), which the
other GPU tests pin to the oracle; B = 1 masked Conv calls take the split
form (the one-column MAC kernel), even B the fused form."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu

T = U.T
# plain-20's four Conv layouts at N = 8192 (2G = 2, 8, 4, 2) and its FC
SHAPES = [dict(ci=3, co=16, h=32, w=32), dict(ci=16, co=16, h=32, w=32), dict(ci=32, co=32, h=16, w=16),
          dict(ci=64, co=64, h=8, w=8)]


def _i32(a):
    torch = U.torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, np.int32).ravel()).cuda()


class _Case:
    """Banks and device buffers of one masked / client / plain layer call."""

    def __init__(self, H, p, N, ps, psis, kind, shape, B, seed, in_ntt=False):
        L = len(ps)
        self.kind, self.shape, self.B = kind, shape, B
        self.dom = H.HE_COEFF
        if shape.get("fc"):
            n_in, n_out = shape["n_in"], shape["n_out"]
            lay = O.fc_layout(N, n_in, n_out)
            G, Hh = 1, lay["P"]
            W = synth.fc_weights(seed, "mpl/W", n_out, n_in, -128, 127)
            bias = synth.ints(seed, "mpl/b", (n_out,), -900, 900).astype(np.int32)
            rho = synth.ints(seed, "mpl/rho", (Hh, N), 0, T - 1).astype(np.uint32)
            pp = (Hh, L, N)
            c0_shape, sh_shape, shp_shape = (B, L, N), (B, N), (B, Hh, N)
        else:
            lay = O.conv_layout(N, shape["ci"], shape["co"], shape["h"], shape["w"])
            G, Hh = lay["G"], lay["H"]
            F = synth.conv_weights(seed, "mpl/F", shape["co"], shape["ci"], 3, 3, -128, 127)
            rho = synth.ints(seed, "mpl/rho", (shape["co"], G, N), 0, T - 1).astype(np.uint32)
            pp = (shape["co"], G, L, N)
            c0_shape, sh_shape, shp_shape = (B, G, L, N), (B, G, N), (B, Hh, N)
        self.out_shape = (B, Hh, L, N) if kind != "plain" else (B, Hh, 2, L, N)
        fc = shape.get("fc")
        if kind == "server":
            self.f = (H.he_pack_fc_masked(p, n_in, n_out, W, bias, rho) if fc
                      else H.he_pack_masked(p, shape, F, rho))
            c0 = synth.residues(seed, "mpl/c0", c0_shape, ps)
            if in_ntt:
                c0 = c0.copy()
                for l in range(L):
                    c0[..., l, :] = O.ntt_fwd(np.ascontiguousarray(c0[..., l, :]), ps[l], psis[l])
                self.dom = H.HE_NTT
            self.d_in = U.to_dev(c0)
            self.d_sh = U.to_dev(synth.ints(seed, "mpl/sh", sh_shape, 0, T - 1).astype(np.uint32))
            self.d_shp = U.to_dev(synth.ints(seed, "mpl/shp", shp_shape, 0, T - 1).astype(np.uint32))
        elif kind == "client":
            p1 = synth.residues(seed, "mpl/p1", pp, ps)
            p2 = synth.residues(seed, "mpl/p2", pp, ps)
            self.f = (H.he_pack_fc_client(p, n_in, n_out, p1, p2) if fc
                      else H.he_pack_client(p, shape, p1, p2))
            self.d_in = _i32(synth.ints(seed, "mpl/v", sh_shape, -1, 1))
            self.d_sh = _i32(synth.ints(seed, "mpl/ish", sh_shape, -8, T + 7))
            self.d_shp = None
        else:
            self.f = H.he_pack_fc(p, n_in, n_out, W, bias) if fc else H.he_pack_filters(p, shape, F)
            cts = synth.residues(seed, "mpl/ct", (B, 2, L, N) if fc else (B, G, 2, L, N), ps)
            self.d_in = U.to_dev(cts)
            self.d_sh = self.d_shp = None
        self.d_out = U.empty_dev(self.out_shape)
        # every form transforms B * (G or 2G) * 2 * L * N / 2 ... words: the
        # most any of them needs is B * 2G * L * N (G = 1 for an FC layer)
        U.reserve(p, B * 2 * G * L * N * 4)

    def call(self):
        return (self.f, self.d_in, self.dom, self.d_out, self.B, self.d_sh, self.d_shp)

    def single(self, H, p, stream):
        d = U.empty_dev(self.out_shape)
        fc = self.shape.get("fc")
        if self.kind == "server":
            (H.he_fc_layer_masked if fc else H.he_conv_layer_masked)(p, self.f, self.d_in, self.d_sh, self.d_shp,
                                                                      self.dom, d, self.B, stream)
        elif self.kind == "client":
            (H.he_fc_client if fc else H.he_conv_client)(p, self.f, self.d_in, self.d_sh, d, self.B, stream)
        else:
            (H.he_fc_layer if fc else H.he_conv_layer)(p, self.f, self.d_in, self.dom, d, H.HE_OUT_EXTRACTED,
                                                       self.B, stream)
        H.he_sync(stream)
        return U.from_dev(d).reshape(self.out_shape)


def _run_plan(H, cases, stream, graph=False, fc_direct=1, fin_parts=1):
    torch = U.torch_cuda()
    plan = H.he_plan_create_tuned([c.call() for c in cases],
                                  dict(H.he_plan_tuning_default(), fc_direct=fc_direct, fin_parts=fin_parts))
    try:
        info = H.he_plan_query(plan, len(cases))
        outs = []
        for rep in range(2):   # every word rewritten on each run
            for c in cases:
                c.d_out.fill_(-1)
            if graph:
                g = torch.cuda.CUDAGraph()
                H.he_plan_run(plan, stream)
                H.he_sync(stream)
                with torch.cuda.graph(g, stream=stream):
                    H.he_plan_run(plan, stream)
                for c in cases:
                    c.d_out.fill_(-1)
                g.replay()
                torch.cuda.synchronize()
            else:
                H.he_plan_run(plan, stream)
                H.he_sync(stream)
            H.he_plan_check(plan)
            outs.append([U.from_dev(c.d_out).reshape(c.out_shape) for c in cases])
        return info, outs
    finally:
        H.he_plan_destroy(plan)


def _mixed(H, p, N, ps, psis, B=1, in_ntt=False):
    cases = []
    for k, shape in enumerate(SHAPES):
        cases.append(_Case(H, p, N, ps, psis, "server", shape, B, 300 + k, in_ntt=in_ntt))
        cases.append(_Case(H, p, N, ps, psis, "client", shape, B, 310 + k))
    fc = dict(fc=True, n_in=64, n_out=10)
    cases.append(_Case(H, p, N, ps, psis, "server", fc, B, 320, in_ntt=in_ntt))
    cases.append(_Case(H, p, N, ps, psis, "client", fc, B, 321))
    cases.append(_Case(H, p, N, ps, psis, "plain", SHAPES[2], B, 322))
    cases.append(_Case(H, p, N, ps, psis, "plain", fc, B, 323))
    return cases


# fc_direct: the FC windows computed directly (2: every coefficient-domain
# FC call, masked and client ones included; 1: the cost rule, which keeps the
# masked and client windows on the transform path) or through the
# transforms; fin_parts: finishing items over 1, 2 or 4 shares of the
# residue classes; the words are the same
@pytest.mark.parametrize("in_ntt,fc_direct,fin_parts", [(False, 2, 1), (True, 1, 2), (False, 0, 4)])
def test_masked_and_client_calls_in_one_plan_match_single_calls(in_ntt, fc_direct, fin_parts):
    H = U.he()
    torch = U.torch_cuda()
    N, L = 8192, 3
    ps, psis = U.ring(N, L)
    s = torch.cuda.current_stream()
    with U.params(N, L) as p:
        cases = _mixed(H, p, N, ps, psis, in_ntt=in_ntt)
        try:
            info, outs = _run_plan(H, cases, s, fc_direct=fc_direct, fin_parts=fin_parts)
            # B = 1 masked and client Conv calls run in the split form
            for i, c in enumerate(cases):
                if c.kind != "plain" and not c.shape.get("fc"):
                    assert info["form"][i] == 1, (i, c.kind, c.shape)
            for c, got in zip(cases, outs[0]):
                np.testing.assert_array_equal(got, c.single(H, p, s), err_msg=f"{c.kind} {c.shape}")
            for a, b in zip(outs[0], outs[1]):
                np.testing.assert_array_equal(a, b)
        finally:
            for c in cases:
                H.he_filters_destroy(c.f)


@pytest.mark.parametrize("fc_direct", [2, 1, 0])
def test_masked_plan_matches_the_oracle(fc_direct):
    """One masked Conv call (16 -> 16 at 32x32: 2G = 8) and one masked FC call
    in a plan, against the oracle's words directly (the FC window computed
    directly, or through the transforms)."""
    H = U.he()
    torch = U.torch_cuda()
    N, L = 8192, 3
    ps, psis = U.ring(N, L)
    s = torch.cuda.current_stream()
    shape = SHAPES[1]
    lay = O.conv_layout(N, shape["ci"], shape["co"], shape["h"], shape["w"])
    G, Hh = lay["G"], lay["H"]
    c0 = synth.residues(5, "mo/c0", (1, G, L, N), ps)
    sh = synth.ints(5, "mo/sh", (1, G, N), 0, T - 1).astype(np.uint32)
    rho = synth.ints(5, "mo/rho", (16, G, N), 0, T - 1).astype(np.uint32)
    shp = synth.ints(5, "mo/shp", (1, Hh, N), 0, T - 1).astype(np.uint32)
    F = synth.conv_weights(5, "mo/F", 16, 16, 3, 3, -128, 127)
    fl = O.fc_layout(N, 64, 10)
    fc0 = synth.residues(6, "mo/fc0", (1, L, N), ps)
    fsh = synth.ints(6, "mo/fsh", (1, N), 0, T - 1).astype(np.uint32)
    frho = synth.ints(6, "mo/frho", (fl["P"], N), 0, T - 1).astype(np.uint32)
    fshp = synth.ints(6, "mo/fshp", (1, fl["P"], N), 0, T - 1).astype(np.uint32)
    W = synth.fc_weights(6, "mo/W", 10, 64, -128, 127)
    bias = synth.ints(6, "mo/b", (10,), -99, 99).astype(np.int32)
    ref = O.conv_layer_masked(c0, sh, rho, F, shp, ps, psis, T, lay, tier="ntt")
    fref = O.fc_layer_masked(fc0, fsh, frho, W, bias, fshp, ps, psis, T, fl, tier="ntt")
    with U.params(N, L) as p:
        f = H.he_pack_masked(p, shape, F, rho)
        ff = H.he_pack_fc_masked(p, 64, 10, W, bias, frho)
        try:
            d_out, fd_out = U.empty_dev(ref.shape), U.empty_dev(fref.shape)
            calls = [(f, U.to_dev(c0), H.HE_COEFF, d_out, 1, U.to_dev(sh), U.to_dev(shp)),
                     (ff, U.to_dev(fc0), H.HE_COEFF, fd_out, 1, U.to_dev(fsh), U.to_dev(fshp))]
            plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), fc_direct=fc_direct))
            try:
                H.he_plan_run(plan, s)
                H.he_sync(s)
                H.he_plan_check(plan)
            finally:
                H.he_plan_destroy(plan)
            np.testing.assert_array_equal(U.from_dev(d_out).reshape(ref.shape), ref)
            np.testing.assert_array_equal(U.from_dev(fd_out).reshape(fref.shape), fref)
        finally:
            H.he_filters_destroy(f)
            H.he_filters_destroy(ff)


def test_batched_masked_calls_take_the_fused_form_and_graph_capture():
    H = U.he()
    torch = U.torch_cuda()
    N, L = 4096, 2
    ps, psis = U.ring(N, L)
    s = torch.cuda.Stream()
    with U.params(N, L) as p:
        # even batches in column tiles of 2 and more, odd ones in tiles of one
        cases = [_Case(H, p, N, ps, psis, "server", SHAPES[2], 2, 330),
                 _Case(H, p, N, ps, psis, "client", SHAPES[3], 4, 331),
                 _Case(H, p, N, ps, psis, "server", dict(fc=True, n_in=100, n_out=40), 3, 332),
                 _Case(H, p, N, ps, psis, "server", SHAPES[1], 3, 333),
                 _Case(H, p, N, ps, psis, "client", SHAPES[2], 5, 334)]
        try:
            with torch.cuda.stream(s):
                info, outs = _run_plan(H, cases, s, graph=True)
            assert info["form"][0] == 0 and info["form"][1] == 0 and info["form"][3] == 0 and info["form"][4] == 0
            for c, got in zip(cases, outs[0]):
                np.testing.assert_array_equal(got, c.single(H, p, s), err_msg=f"{c.kind} {c.shape}")
        finally:
            for c in cases:
                H.he_filters_destroy(c.f)


def test_masked_plan_argument_errors():
    H = U.he()
    N, L = 4096, 2
    ps, psis = U.ring(N, L)
    with U.params(N, L) as p:
        c1 = _Case(H, p, N, ps, psis, "server", SHAPES[2], 1, 341)
        cc = _Case(H, p, N, ps, psis, "client", SHAPES[2], 1, 342)
        try:
            with pytest.raises(RuntimeError):                        # a client call with NTT-domain inputs
                H.he_plan_create([(cc.f, cc.d_in, H.HE_NTT, cc.d_out, 1, cc.d_sh)])
            with pytest.raises(RuntimeError):                        # no shares
                H.he_plan_create([(c1.f, c1.d_in, H.HE_COEFF, c1.d_out, 1)])
            with pytest.raises(RuntimeError):                        # output overlapping a share
                H.he_plan_create([(c1.f, c1.d_in, H.HE_COEFF, c1.d_sh, 1, c1.d_sh, c1.d_shp)])
        finally:
            H.he_filters_destroy(c1.f)
            H.he_filters_destroy(cc.f)
